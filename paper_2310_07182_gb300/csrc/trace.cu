// trace.cu -- closest-hit BVH traversal (the intersection step, which dominates path
// tracing time, Sec. 1), one ray per thread.
//
// Stackful while-while traversal of the 64-byte two-child nodes: both child boxes are
// fetched with four 16-byte read-only loads, tested with a conservative slab test, the
// nearer hit child is visited first and the farther one pushed.  The traversal stack lives
// in shared memory (kSmemStack entries per thread, interleaved so that a warp's pushes hit
// distinct banks) and continues in a per-thread local array for deeper trees.  Leaves hold
// up to four triangles tested with the watertight test of Woop, Benthin and Wald (2013).
//
// Closest-hit rule, identical for the BVH2 and BVH8-Q kernels (the BVH8-Q kernel is below): accept t > 0 if
// t < t_best, or t == t_best and the original triangle index is smaller.  Boxes are culled
// only if their entry distance exceeds t_best (1 + 2^-16) and the slab exit is widened by
// (1 + 2^-21) > 1 + 2 gamma_3 (Ize 2013), so no box that holds a candidate triangle is ever
// skipped and both BVH layouts return the same hit bit for bit.
#include <cuda_runtime.h>

#include "cr_internal.h"

namespace cr {
namespace {

constexpr int kSmemStack = 16;  // entries per thread in shared memory
constexpr int kStackTotal = 64; // >= BVH depth (the builder keeps depth <= 64)
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
// first kSmemStack entries in shared memory, the rest in a local array
#define STACK_PUSH(v)                                                                \
    do {                                                                             \
        if (sp < kSmemStack) sstack[sp * stride] = (uint32_t)(v);                    \
        else if (sp < kStackTotal) lstack[sp - kSmemStack] = (v);                   \
        sp = sp < kStackTotal ? sp + 1 : sp; /* the builder keeps depth < kStackTotal */ \
    } while (0)
#define STACK_POP(v)                                                                 \
    do {                                                                             \
        --sp;                                                                        \
        (v) = sp < kSmemStack ? (int)sstack[sp * stride] : lstack[sp - kSmemStack]; \
    } while (0)
#endif

// kAny: visibility only; the traversal ends at the first triangle hit before the ray's tmax.
template <bool kCount, bool kAny = false>
__device__ __forceinline__ int2 trace_bvh2_one(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                               float4 ro, float4 rd, uint32_t* sstack, unsigned long long& n_node,
                                               unsigned long long& n_tri) {
    const RayPre r = prep_ray(ro, rd);
    const int skip = __float_as_int(ro.w);
    Best best{rd.w, -1, 0x7fffffff};
#if CR_TRACE_LOCAL_STACK
    int lstack_all[kStackTotal];
    (void)sstack;
#else
    int lstack[kStackTotal - kSmemStack];
    const int stride = blockDim.x;
#endif
    int sp = 0;
    int node = 0;
    while (true) {
        while (node >= 0) {
            if (kCount) ++n_node;
            const float4 n0 = __ldg(&nodes[4 * node + 0]);
            const float4 n1 = __ldg(&nodes[4 * node + 1]);
            const float4 n2 = __ldg(&nodes[4 * node + 2]);
            const float4 n3 = __ldg(&nodes[4 * node + 3]);
            const float tcull = __fmul_rn(best.t, kCullWiden);
            const float t0 = box_entry_fma(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tcull);
            const float t1 = box_entry_fma(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tcull);
            const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            const bool h0 = t0 != INFINITY, h1 = t1 != INFINITY;
            if (h0 && h1) {
                const bool first0 = t0 <= t1;
                const int near = first0 ? c0 : c1, far = first0 ? c1 : c0;
                STACK_PUSH(far);
                node = near;
            } else if (h0 || h1) {
                node = h0 ? c0 : c1;
            } else {
                if (sp == 0) { node = 0x7fffffff; break; }
                STACK_POP(node);
            }
        }
        if (node == 0x7fffffff) break;
        // leaf
        const uint32_t code = (uint32_t)(~node);
        test_leaf(tris, r, skip, code >> 2, (code & 3u) + 1u, best, n_tri);
        if (kAny && best.leaf >= 0) break;
        if (sp == 0) break;
        STACK_POP(node);
    }
    return make_int2(best.leaf, __float_as_int(best.t));
}

#ifndef CR_TRACE_MAXNREG
#define CR_TRACE_MAXNREG 48 // caps registers so 10 blocks of 128 threads stay resident per SM
#endif

template <bool kCount, bool kAny = false>
__global__ void __maxnreg__(CR_TRACE_MAXNREG) k_trace_bvh2(const SceneDev* __restrict__ scenes, const uint16_t* __restrict__ slot_scene,
                             const float4* __restrict__ ray_o, const float4* __restrict__ ray_d,
                             const int32_t* __restrict__ queue, const uint32_t* __restrict__ queue_count,
                             uint32_t n_max, int2* __restrict__ hit, unsigned long long* counters) {
    extern __shared__ uint32_t smem_stack[];
    const uint32_t n = queue_count ? min(*queue_count, n_max) : n_max;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long n_node = 0, n_tri = 0;
    if (i < n) {
        const int slot = queue ? queue[i] : (int)i;
        const SceneDev& sc = scenes[slot_scene ? slot_scene[slot] : 0];
        const float4 ro = ray_o[slot];
        const float4 rd = ray_d[slot];
        int2 h = make_int2(-1, __float_as_int(INFINITY));
        if (rd.w >= 0.0f)
            h = trace_bvh2_one<kCount, kAny>(sc.nodes2, sc.tris, ro, rd, smem_stack + threadIdx.x, n_node, n_tri);
        hit[slot] = h;
    }
    if (kCount) {
        for (int off = 16; off > 0; off >>= 1) {
            n_node += __shfl_down_sync(0xffffffffu, n_node, off);
            n_tri += __shfl_down_sync(0xffffffffu, n_tri, off);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&counters[0], n_node);
            atomicAdd(&counters[1], n_tri);
        }
    }
}

// Two-phase variant: phase 1 traverses every ray for at most `budget` node and leaf visits;
// a ray that runs out saves its traversal state (next node, stack, best hit) and is flagged.
// The flagged rays are compacted in queue order (so neighbours stay neighbours) and phase 2
// resumes them in full warps, so short rays no longer leave most lanes of a warp idle while
// its long rays finish.  Suspension only happens with at most kSaveStack entries on the
// stack (deeper rays run to completion in phase 1).  The visit order is the single-ray
// kernel's, so the hits are identical.
constexpr int kSaveStack = 24;

__device__ __forceinline__ int2 trace_bvh2_resumable(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                                     float4 ro, float4 rd, uint32_t* sstack, uint32_t budget,
                                                     TraceState* st, bool resume, bool& suspended) {
    const RayPre r = prep_ray(ro, rd);
    const int skip = __float_as_int(ro.w);
    Best best{rd.w, -1, 0x7fffffff};
    int lstack[kStackTotal - kSmemStack];
    const int stride = blockDim.x;
    int sp = 0, node = 0;
    if (resume) {
        node = st->node;
        sp = st->sp;
        best = Best{st->t, st->leaf, st->orig};
        for (int k = 0; k < sp; ++k) {
            const int v = st->stack[k];
            if (k < kSmemStack) sstack[k * stride] = (uint32_t)v;
            else lstack[k - kSmemStack] = v;
        }
    }
    uint32_t visits = 0;
    suspended = false;
    while (true) {
        while (node >= 0) {
            if (++visits > budget && sp <= kSaveStack) {
                suspended = true;
                break;
            }
            const float4 n0 = __ldg(&nodes[4 * node + 0]);
            const float4 n1 = __ldg(&nodes[4 * node + 1]);
            const float4 n2 = __ldg(&nodes[4 * node + 2]);
            const float4 n3 = __ldg(&nodes[4 * node + 3]);
            const float tcull = __fmul_rn(best.t, kCullWiden);
            const float t0 = box_entry_fma(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tcull);
            const float t1 = box_entry_fma(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tcull);
            const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            const bool h0 = t0 != INFINITY, h1 = t1 != INFINITY;
            if (h0 && h1) {
                const bool first0 = t0 <= t1;
                const int near = first0 ? c0 : c1, far = first0 ? c1 : c0;
                STACK_PUSH(far);
                node = near;
            } else if (h0 || h1) {
                node = h0 ? c0 : c1;
            } else {
                if (sp == 0) { node = 0x7fffffff; break; }
                STACK_POP(node);
            }
        }
        if (suspended || node == 0x7fffffff) break;
        const uint32_t code = (uint32_t)(~node);
        unsigned long long dummy = 0;
        test_leaf(tris, r, skip, code >> 2, (code & 3u) + 1u, best, dummy);
        ++visits;
        if (sp == 0) break;
        STACK_POP(node);
    }
    if (suspended) {
        st->node = node;
        st->sp = sp;
        st->t = best.t;
        st->leaf = best.leaf;
        st->orig = best.orig;
        for (int k = 0; k < sp; ++k) st->stack[k] = k < kSmemStack ? (int)sstack[k * stride] : lstack[k - kSmemStack];
    }
    return make_int2(best.leaf, __float_as_int(best.t));
}

__global__ void __maxnreg__(CR_TRACE_MAXNREG) k_trace_bvh2_phase(
    const SceneDev* __restrict__ scenes, const uint16_t* __restrict__ slot_scene, const float4* __restrict__ ray_o,
    const float4* __restrict__ ray_d, const int32_t* __restrict__ queue, const uint32_t* __restrict__ queue_count,
    uint32_t n_max, int2* __restrict__ hit, TraceState* __restrict__ state, uint8_t* __restrict__ susp,
    uint32_t budget, int resume) {
    extern __shared__ uint32_t smem_stack[];
    const uint32_t n = queue_count ? min(*queue_count, n_max) : n_max;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int slot = queue ? queue[i] : (int)i;
    const float4 ro = ray_o[slot];
    const float4 rd = ray_d[slot];
    bool suspended = false;
    int2 h = make_int2(-1, __float_as_int(INFINITY));
    if (rd.w >= 0.0f) {
        const SceneDev& sc = scenes[slot_scene ? slot_scene[slot] : 0];
        h = trace_bvh2_resumable(sc.nodes2, sc.tris, ro, rd, smem_stack + threadIdx.x, budget, &state[slot],
                                 resume != 0, suspended);
    }
    if (!suspended) hit[slot] = h;
    if (susp) susp[i] = suspended ? 1 : 0;
}

// Order-preserving compaction of the suspended rays' queue entries (count, scan, scatter).
__global__ void __launch_bounds__(256) k_susp_count(const uint8_t* __restrict__ susp, const uint32_t* __restrict__ count,
                                                    uint32_t n_max, uint32_t* __restrict__ block_counts) {
    __shared__ uint32_t s_w[8];
    const uint32_t n = min(*count, n_max);
    const uint32_t i = blockIdx.x * 256 + threadIdx.x;
    const uint32_t f = (i < n && susp[i]) ? 1u : 0u;
    const uint32_t b = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        block_counts[2 * blockIdx.x] = t;
        block_counts[2 * blockIdx.x + 1] = 0;
    }
}

__global__ void __launch_bounds__(256) k_susp_scatter(const uint8_t* __restrict__ susp, const int32_t* __restrict__ queue,
                                                      const uint32_t* __restrict__ count, uint32_t n_max,
                                                      const uint32_t* __restrict__ block_offsets,
                                                      int32_t* __restrict__ out_queue) {
    __shared__ uint32_t s_w[8];
    const uint32_t n = min(*count, n_max);
    const uint32_t i = blockIdx.x * 256 + threadIdx.x;
    const uint32_t f = (i < n && susp[i]) ? 1u : 0u;
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t b = __ballot_sync(0xffffffffu, f);
    if (lane == 0) s_w[w] = __popc(b);
    __syncthreads();
    uint32_t before = 0;
    for (uint32_t k = 0; k < w; ++k) before += s_w[k];
    if (f) out_queue[block_offsets[2 * blockIdx.x] + before + __popc(b & ((1u << lane) - 1u))] = queue[i];
}

// Warp-packet variant: the 32 lanes of a warp traverse ONE node sequence.  At each inner
// node every lane tests both child boxes against its own ray (with its own culling
// distance); a child is entered if any lane's ray reaches it, nearer-first by majority.
// Leaves are tested by every lane against its own ray.  Each lane therefore visits a
// superset of the boxes its own ray enters, with the same triangle test and tie rule, so
// the hits are the single-ray kernel's bit for bit.  Control flow is warp-uniform, which
// pays off when the rays of a warp are coherent (primary rays, reused directions) and
// costs extra box and triangle tests when they are not.
__global__ void __maxnreg__(CR_TRACE_MAXNREG) k_trace_bvh2_packet(
    const SceneDev* __restrict__ scenes, const uint16_t* __restrict__ slot_scene, const float4* __restrict__ ray_o,
    const float4* __restrict__ ray_d, const int32_t* __restrict__ queue, const uint32_t* __restrict__ queue_count,
    uint32_t n_max, int2* __restrict__ hit) {
    extern __shared__ uint32_t smem_stack[];
    uint32_t* sstack = smem_stack + threadIdx.x;
    const int stride = blockDim.x;
    const uint32_t n = queue_count ? min(*queue_count, n_max) : n_max;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (__all_sync(0xffffffffu, i >= n)) return;
    int slot = -1;
    bool valid = false;
    RayPre r;
    int skip = -1;
    Best best{-1.0f, -1, 0x7fffffff}; // t < 0: a lane without a ray never enters a box
    uint32_t sid = 0;
    if (i < n) {
        slot = queue ? queue[i] : (int)i;
        const float4 ro = ray_o[slot];
        const float4 rd = ray_d[slot];
        sid = slot_scene ? slot_scene[slot] : 0;
        if (rd.w >= 0.0f) {
            r = prep_ray(ro, rd);
            skip = __float_as_int(ro.w);
            best = Best{rd.w, -1, 0x7fffffff};
            valid = true;
        } else {
            hit[slot] = make_int2(-1, __float_as_int(INFINITY));
        }
    }
    // a warp shares one scene (slots of one tile are one job); mixed warps take the slow path
    const uint32_t sid0 = __shfl_sync(0xffffffffu, sid, 0);
    const bool uniform_scene = __all_sync(0xffffffffu, !valid || sid == sid0);
    const SceneDev& sc = scenes[uniform_scene ? sid0 : sid];
    const float4* nodes = sc.nodes2;
    const float4* tris = sc.tris;
    unsigned long long dummy = 0;
    if (!uniform_scene) { // rare: a warp straddling two jobs of different scenes
        if (valid) {
            int2 h = trace_bvh2_one<false>(nodes, tris, ray_o[slot], ray_d[slot], sstack, dummy, dummy);
            hit[slot] = h;
        }
        return;
    }
#if CR_TRACE_LOCAL_STACK
    int lstack_all[kStackTotal];
#else
    int lstack[kStackTotal - kSmemStack];
#endif
    int sp = 0;
    int node = 0;
    if (!valid) r = prep_ray(make_float4(0, 0, 0, 0), make_float4(0, 0, 1, -1)); // inert ray
    while (true) {
        if (node >= 0) {
            const float4 n0 = __ldg(&nodes[4 * node + 0]);
            const float4 n1 = __ldg(&nodes[4 * node + 1]);
            const float4 n2 = __ldg(&nodes[4 * node + 2]);
            const float4 n3 = __ldg(&nodes[4 * node + 3]);
            const float tcull = __fmul_rn(best.t, kCullWiden); // negative for lanes without a ray
            const float t0 = box_entry_fma(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tcull);
            const float t1 = box_entry_fma(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tcull);
            const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            const bool h0 = t0 != INFINITY, h1 = t1 != INFINITY;
            const uint32_t v0 = __ballot_sync(0xffffffffu, h0 && (!h1 || t0 <= t1));
            const uint32_t v1 = __ballot_sync(0xffffffffu, h1 && (!h0 || t1 < t0));
            const bool any0 = __any_sync(0xffffffffu, h0), any1 = __any_sync(0xffffffffu, h1);
            if (any0 && any1) {
                const bool first0 = __popc(v0) >= __popc(v1);
                STACK_PUSH(first0 ? c1 : c0);
                node = first0 ? c0 : c1;
                continue;
            } else if (any0 || any1) {
                node = any0 ? c0 : c1;
                continue;
            }
        } else {
            const uint32_t code = (uint32_t)(~node);
            if (valid) test_leaf(tris, r, skip, code >> 2, (code & 3u) + 1u, best, dummy);
        }
        if (sp == 0) break;
        STACK_POP(node);
    }
    if (valid) hit[slot] = make_int2(best.leaf, __float_as_int(best.t));
}

// Speculative variant: lanes keep one reached leaf pending and go on descending inner
// nodes until every lane of the warp holds a leaf or has finished; then all lanes test
// their pending leaves together.  Inner-node and leaf phases thus run with more active
// lanes.  The loops are warp-synchronous: every lane (finished or not) executes each
// iteration, and every iteration either visits a node, parks a leaf or tests one.
constexpr int kEmpty = 0x7fffffff; // stack exhausted

__global__ void __maxnreg__(CR_TRACE_MAXNREG) k_trace_bvh2_spec(
    const SceneDev* __restrict__ scenes, const uint16_t* __restrict__ slot_scene, const float4* __restrict__ ray_o,
    const float4* __restrict__ ray_d, const int32_t* __restrict__ queue, const uint32_t* __restrict__ queue_count,
    uint32_t n_max, int2* __restrict__ hit) {
    extern __shared__ uint32_t smem_stack[];
    uint32_t* sstack = smem_stack + threadIdx.x;
    const int stride = blockDim.x;
    const uint32_t n = queue_count ? min(*queue_count, n_max) : n_max;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    // whole warps past the end leave together; the others run every iteration
    if (__all_sync(0xffffffffu, i >= n)) return;
    int slot = -1;
    bool done = true;
    RayPre r;
    int skip = -1;
    Best best{0.0f, -1, 0x7fffffff};
    const float4* nodes = nullptr;
    const float4* tris = nullptr;
    if (i < n) {
        slot = queue ? queue[i] : (int)i;
        const float4 ro = ray_o[slot];
        const float4 rd = ray_d[slot];
        if (rd.w >= 0.0f) {
            const SceneDev& sc = scenes[slot_scene ? slot_scene[slot] : 0];
            nodes = sc.nodes2;
            tris = sc.tris;
            r = prep_ray(ro, rd);
            skip = __float_as_int(ro.w);
            best = Best{rd.w, -1, 0x7fffffff};
            done = false;
        } else {
            hit[slot] = make_int2(-1, __float_as_int(INFINITY));
        }
    }
    int lstack[kStackTotal - kSmemStack];
    int sp = 0, node = done ? kEmpty : 0, leaf = 0;
    unsigned long long dummy = 0;
    auto pop = [&]() -> int {
        if (sp == 0) return kEmpty;
        --sp;
        return sp < kSmemStack ? (int)sstack[sp * stride] : lstack[sp - kSmemStack];
    };
    while (true) {
        // inner phase
        while (true) {
            if (node >= 0 && node != kEmpty) {
                const float4 n0 = __ldg(&nodes[4 * node + 0]);
                const float4 n1 = __ldg(&nodes[4 * node + 1]);
                const float4 n2 = __ldg(&nodes[4 * node + 2]);
                const float4 n3 = __ldg(&nodes[4 * node + 3]);
                const float tcull = __fmul_rn(best.t, kCullWiden);
                const float t0 = box_entry_fma(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tcull);
                const float t1 = box_entry_fma(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tcull);
                const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
                const bool h0 = t0 != INFINITY, h1 = t1 != INFINITY;
                if (h0 && h1) {
                    const bool first0 = t0 <= t1;
                    const int far = first0 ? c1 : c0;
                    node = first0 ? c0 : c1;
                    if (sp < kSmemStack) sstack[sp * stride] = (uint32_t)far;
                    else if (sp < kStackTotal) lstack[sp - kSmemStack] = far;
                    sp = sp < kStackTotal ? sp + 1 : sp; // the builder keeps depth < kStackTotal
                } else if (h0 || h1) {
                    node = h0 ? c0 : c1;
                } else {
                    node = pop();
                }
            }
            if (node < 0 && leaf == 0) { // park the reached leaf and keep descending
                leaf = node;
                node = pop();
            }
            const bool searching = leaf == 0 && node != kEmpty;
            if (!__any_sync(0xffffffffu, searching)) break;
        }
        // leaf phase: the parked leaf, then any leaf the descent stopped on
        while (leaf < 0) {
            const uint32_t code = (uint32_t)(~leaf);
            test_leaf(tris, r, skip, code >> 2, (code & 3u) + 1u, best, dummy);
            leaf = 0;
            if (node < 0) {
                leaf = node;
                node = pop();
            }
        }
        if (!done && node == kEmpty) {
            hit[slot] = make_int2(best.leaf, __float_as_int(best.t));
            done = true;
        }
        if (__all_sync(0xffffffffu, done)) break;
    }
}

// Persistent variant with dynamic ray fetch: a fixed grid of resident blocks whose warps keep
// every lane busy.  A lane that finishes its ray takes the next one from its warp's chunk
// of the queue (the warp grabs kChunk rays at a time with one atomic), once at least
// `refill` lanes of the warp are idle.  Rays of very different traversal lengths then no
// longer hold a warp until the slowest one ends.  Each lane advances one leaf at a time, so
// idle lanes are refilled between leaves.  Every loop iteration either advances a live
// ray or takes rays from the counter, which only grows, so the loop ends.
constexpr uint32_t kChunk = 256;
constexpr int kDone = 0x7fffffff;

__global__ void __launch_bounds__(128) k_trace_bvh2_dynamic(
    const SceneDev* __restrict__ scenes, const uint16_t* __restrict__ slot_scene, const float4* __restrict__ ray_o,
    const float4* __restrict__ ray_d, const int32_t* __restrict__ queue, const uint32_t* __restrict__ queue_count,
    uint32_t n_max, int2* __restrict__ hit, uint32_t* work, uint32_t refill) {
    extern __shared__ uint32_t smem_stack[];
    uint32_t* sstack = smem_stack + threadIdx.x;
    const int stride = blockDim.x;
    const uint32_t n = queue_count ? min(*queue_count, n_max) : n_max;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t chunk_next = 0, chunk_end = 0; // warp-uniform
    bool exhausted = false;                 // warp-uniform
    bool live = false;
    RayPre r;
    int skip = -1, node = kDone, sp = 0, slot = -1;
    const float4* nodes = nullptr;
    const float4* tris = nullptr;
    Best best{0.0f, -1, 0x7fffffff};
    int lstack[kStackTotal - kSmemStack];
    unsigned long long dummy = 0;
    while (true) {
        uint32_t idle = ~__ballot_sync(0xffffffffu, live);
        if (!exhausted && (uint32_t)__popc(idle) >= refill) {
            if (chunk_next >= chunk_end) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(work, kChunk);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= n) {
                    exhausted = true;
                } else {
                    chunk_next = base;
                    chunk_end = min(base + kChunk, n);
                }
            }
            if (!exhausted) {
                const uint32_t avail = chunk_end - chunk_next;
                const uint32_t k = (uint32_t)__popc(idle);
                if (!live) {
                    const uint32_t rank = __popc(idle & lt_mask);
                    if (rank < avail) {
                        const uint32_t i = chunk_next + rank;
                        slot = queue ? queue[i] : (int)i;
                        const float4 ro = ray_o[slot];
                        const float4 rd = ray_d[slot];
                        if (rd.w >= 0.0f) {
                            const SceneDev& sc = scenes[slot_scene ? slot_scene[slot] : 0];
                            nodes = sc.nodes2;
                            tris = sc.tris;
                            r = prep_ray(ro, rd);
                            skip = __float_as_int(ro.w);
                            best = Best{rd.w, -1, 0x7fffffff};
                            node = 0;
                            sp = 0;
                            live = true;
                        } else {
                            hit[slot] = make_int2(-1, __float_as_int(INFINITY));
                        }
                    }
                }
                chunk_next += min(avail, k);
            }
            idle = ~__ballot_sync(0xffffffffu, live);
        }
        if (idle == 0xffffffffu) {
            if (exhausted) break;
            continue;
        }
        if (live) {
            // inner nodes until a leaf is reached or the traversal ends
            while (node >= 0 && node != kDone) {
                const float4 n0 = __ldg(&nodes[4 * node + 0]);
                const float4 n1 = __ldg(&nodes[4 * node + 1]);
                const float4 n2 = __ldg(&nodes[4 * node + 2]);
                const float4 n3 = __ldg(&nodes[4 * node + 3]);
                const float tcull = __fmul_rn(best.t, kCullWiden);
                const float t0 = box_entry_fma(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tcull);
                const float t1 = box_entry_fma(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tcull);
                const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
                const bool h0 = t0 != INFINITY, h1 = t1 != INFINITY;
                if (h0 && h1) {
                    const bool first0 = t0 <= t1;
                    const int near = first0 ? c0 : c1, far = first0 ? c1 : c0;
                    if (sp < kSmemStack) sstack[sp * stride] = (uint32_t)far;
                    else if (sp < kStackTotal) lstack[sp - kSmemStack] = far;
                    sp = sp < kStackTotal ? sp + 1 : sp; // the builder keeps depth < kStackTotal
                    node = near;
                } else if (h0 || h1) {
                    node = h0 ? c0 : c1;
                } else if (sp == 0) {
                    node = kDone;
                } else {
                    --sp;
                    node = sp < kSmemStack ? (int)sstack[sp * stride] : lstack[sp - kSmemStack];
                }
            }
            if (node != kDone) { // a leaf
                const uint32_t code = (uint32_t)(~node);
                test_leaf(tris, r, skip, code >> 2, (code & 3u) + 1u, best, dummy);
                if (sp == 0) {
                    node = kDone;
                } else {
                    --sp;
                    node = sp < kSmemStack ? (int)sstack[sp * stride] : lstack[sp - kSmemStack];
                }
            }
            if (node == kDone) {
                hit[slot] = make_int2(best.leaf, __float_as_int(best.t));
                live = false;
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// BVH8-Q traversal.  Per node: the 80-byte node is fetched with five 16-byte loads, the valid
// children are decoded (origin + q * step, exact product, one rounded add) and tested with the
// same conservative slab test as the BVH2 kernel, visiting slots in the order k ^ octant(d)
// so that near children tend to come first.  Hit children are pushed far to near except the
// nearest, which is visited next.  Stack entries: inner node index (>= 0) or leaf
// ~((first triangle << 3) | (count - 1)).  Triangles are the BVH8 copy (same records).
constexpr int kStack8 = (int)kBvh8StackCapacity; // >= the builder's stack bound (checked at scene creation)

__device__ __forceinline__ uint32_t byte_of(uint32_t lo, uint32_t hi, uint32_t slot) {
    return ((slot < 4 ? lo : hi) >> (8 * (slot & 3))) & 0xffu;
}

template <bool kCount, bool kAny = false>
__device__ __forceinline__ int2 trace_bvh8_one(const uint4* __restrict__ nodes, const float4* __restrict__ tris,
                                               float4 ro, float4 rd, uint32_t* sstack, unsigned long long& n_node,
                                               unsigned long long& n_tri) {
    const RayPre r = prep_ray(ro, rd);
    const int skip = __float_as_int(ro.w);
    const uint32_t oct = (rd.x < 0.0f ? 1u : 0u) | (rd.y < 0.0f ? 2u : 0u) | (rd.z < 0.0f ? 4u : 0u);
    Best best{rd.w, -1, 0x7fffffff};
    int lstack[kStack8 - kSmemStack];
    int sp = 0;
    int entry = 0;
    const int stride = blockDim.x;
    while (true) {
        if (entry >= 0) {
            if (kCount) ++n_node;
            const uint4 w0 = __ldg(&nodes[5 * entry + 0]);
            const uint4 w1 = __ldg(&nodes[5 * entry + 1]);
            const uint4 w2 = __ldg(&nodes[5 * entry + 2]);
            const uint4 w3 = __ldg(&nodes[5 * entry + 3]);
            const uint4 w4 = __ldg(&nodes[5 * entry + 4]);
            const float ox = __uint_as_float(w0.x), oy = __uint_as_float(w0.y), oz = __uint_as_float(w0.z);
            const float sx = __uint_as_float((w0.w & 0xffu) << 23);
            const float sy = __uint_as_float(((w0.w >> 8) & 0xffu) << 23);
            const float sz = __uint_as_float(((w0.w >> 16) & 0xffu) << 23);
            const uint32_t imask = w0.w >> 24;
            const float tcull = __fmul_rn(best.t, kCullWiden);
            int next = kDone;
#pragma unroll 1
            for (int k = 7; k >= 0; --k) {
                const uint32_t sl = (uint32_t)k ^ oct;
                const uint32_t m = byte_of(w1.z, w1.w, sl);
                const bool inner = (imask >> sl) & 1u;
                if (!inner && m < 32u) continue; // empty slot
                const float lox = __fadd_rn(ox, __fmul_rn((float)byte_of(w2.x, w2.y, sl), sx));
                const float loy = __fadd_rn(oy, __fmul_rn((float)byte_of(w2.z, w2.w, sl), sy));
                const float loz = __fadd_rn(oz, __fmul_rn((float)byte_of(w3.x, w3.y, sl), sz));
                const float hix = __fadd_rn(ox, __fmul_rn((float)byte_of(w3.z, w3.w, sl), sx));
                const float hiy = __fadd_rn(oy, __fmul_rn((float)byte_of(w4.x, w4.y, sl), sy));
                const float hiz = __fadd_rn(oz, __fmul_rn((float)byte_of(w4.z, w4.w, sl), sz));
                if (box_entry(r, lox, hix, loy, hiy, loz, hiz, tcull) == INFINITY) continue;
                const int e = inner ? (int)(w1.x + m) : ~(int)(((w1.y + (m & 31u)) << 3) | ((m >> 5) - 1u));
                if (next != kDone) {
                    if (sp < kSmemStack) sstack[sp * stride] = (uint32_t)next;
                    else if (sp < kStack8) lstack[sp - kSmemStack] = next;
                    sp = sp < kStack8 ? sp + 1 : sp; // scene creation checks the bound
                }
                next = e;
            }
            if (next != kDone) {
                entry = next;
                continue;
            }
        } else {
            const uint32_t code = (uint32_t)(~entry);
            test_leaf(tris, r, skip, code >> 3, (code & 7u) + 1u, best, n_tri);
            if (kAny && best.leaf >= 0) break;
        }
        if (sp == 0) break;
        --sp;
        entry = sp < kSmemStack ? (int)sstack[sp * stride] : lstack[sp - kSmemStack];
    }
    return make_int2(best.leaf, __float_as_int(best.t));
}

template <bool kCount, bool kAny = false>
__global__ void __launch_bounds__(128, 8) k_trace_bvh8(const SceneDev* __restrict__ scenes,
                             const uint16_t* __restrict__ slot_scene,
                             const float4* __restrict__ ray_o, const float4* __restrict__ ray_d,
                             const int32_t* __restrict__ queue, const uint32_t* __restrict__ queue_count,
                             uint32_t n_max, int2* __restrict__ hit, unsigned long long* counters) {
    extern __shared__ uint32_t smem_stack[];
    const uint32_t n = queue_count ? min(*queue_count, n_max) : n_max;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long n_node = 0, n_tri = 0;
    if (i < n) {
        const int slot = queue ? queue[i] : (int)i;
        const SceneDev& sc = scenes[slot_scene ? slot_scene[slot] : 0];
        const float4 ro = ray_o[slot];
        const float4 rd = ray_d[slot];
        int2 h = make_int2(-1, __float_as_int(INFINITY));
        if (rd.w >= 0.0f)
            h = trace_bvh8_one<kCount, kAny>(sc.nodes8, sc.tris, ro, rd, smem_stack + threadIdx.x, n_node, n_tri);
        hit[slot] = h;
    }
    if (kCount) {
        for (int off = 16; off > 0; off >>= 1) {
            n_node += __shfl_down_sync(0xffffffffu, n_node, off);
            n_tri += __shfl_down_sync(0xffffffffu, n_tri, off);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&counters[0], n_node);
            atomicAdd(&counters[1], n_tri);
        }
    }
}

// Shadow rays of next-event estimation, one thread per position of the last shade's group
// queue (so a reuse group's rays run in adjacent lanes, as they were shaded).  A ray whose
// direction record has w = tmax > 0 is traced for visibility only; if nothing blocks it, its
// contribution is added to the path radiance of its slot.  Rays traced are counted.
template <bool kBvh8>
__global__ void __maxnreg__(CR_TRACE_MAXNREG) k_trace_shadow(
    const SceneDev* __restrict__ scenes, const uint16_t* __restrict__ slot_scene, const float4* __restrict__ sh_o,
    const float4* __restrict__ sh_d, const float4* __restrict__ sh_c, const int32_t* __restrict__ group_queue,
    const uint32_t* __restrict__ group_count, uint32_t n_groups_max, uint32_t K, float4* __restrict__ radiance,
    unsigned long long* __restrict__ n_traced) {
    extern __shared__ uint32_t smem_stack[];
    const uint32_t n_groups = group_queue ? min(*group_count, n_groups_max) : n_groups_max;
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    bool traced = false;
    if (pos < n_groups * K) {
        const uint32_t g = group_queue ? (uint32_t)group_queue[pos / K] : pos / K;
        const int slot = (int)(g * K + pos % K);
        const float4 rd = sh_d[slot];
        if (rd.w > 0.0f) {
            traced = true;
            const float4 ro = sh_o[slot];
            const SceneDev& sc = scenes[slot_scene[slot]];
            unsigned long long dn = 0, dt = 0;
            const int2 h = kBvh8 ? trace_bvh8_one<false, true>(sc.nodes8, sc.tris, ro, rd, smem_stack + threadIdx.x, dn, dt)
                                 : trace_bvh2_one<false, true>(sc.nodes2, sc.tris, ro, rd, smem_stack + threadIdx.x, dn, dt);
            if (h.x < 0) {
                const float4 c = sh_c[slot];
                const float4 L = radiance[slot];
                radiance[slot] = make_float4(__fadd_rn(L.x, c.x), __fadd_rn(L.y, c.y), __fadd_rn(L.z, c.z), L.w);
            }
        }
    }
    const uint32_t b = __ballot_sync(0xffffffffu, traced);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_traced, (unsigned long long)__popc(b));
}


__global__ void k_hits_to_user(const float4* __restrict__ tris, const int2* __restrict__ hit, uint32_t n,
                               int32_t* __restrict__ prim, float* __restrict__ t) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 h = hit[i];
    prim[i] = h.x >= 0 ? __float_as_int(__ldg(&tris[3 * h.x]).w) : -1;
    t[i] = h.x >= 0 ? __int_as_float(h.y) : INFINITY; // a miss of a bounded ray reports inf, not tmax
}

__global__ void k_rays_from_user(const float* __restrict__ rays, const int32_t* __restrict__ skip, uint32_t n,
                                 float4* __restrict__ ray_o, float4* __restrict__ ray_d) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* r = rays + 8 * (size_t)i;
    ray_o[i] = make_float4(r[0], r[1], r[2], __int_as_float(skip ? skip[i] : -1));
    ray_d[i] = make_float4(r[4], r[5], r[6], r[7]);
}

} // namespace

void launch_shadow_rays(const SceneDev* scenes, const uint16_t* slot_scene, const float4* sh_o, const float4* sh_d,
                        const float4* sh_c, const int32_t* group_queue, const uint32_t* group_count,
                        uint32_t n_groups_max, uint32_t K, float4* radiance, unsigned long long* n_traced, bool bvh8,
                        cudaStream_t st, LaunchCount& lc) {
    const uint32_t n_pos = n_groups_max * K;
    if (n_pos == 0) return;
    const int block = 128;
    const size_t smem = (size_t)kSmemStack * block * sizeof(uint32_t);
    const uint32_t grid = (n_pos + block - 1) / block;
    if (bvh8)
        k_trace_shadow<true><<<grid, block, smem, st>>>(scenes, slot_scene, sh_o, sh_d, sh_c, group_queue, group_count,
                                                        n_groups_max, K, radiance, n_traced);
    else
        k_trace_shadow<false><<<grid, block, smem, st>>>(scenes, slot_scene, sh_o, sh_d, sh_c, group_queue, group_count,
                                                         n_groups_max, K, radiance, n_traced);
    lc.n++;
}

void launch_rays_from_user(const float* rays, const int32_t* skip, uint32_t n, float4* ray_o, float4* ray_d,
                           cudaStream_t st, LaunchCount& lc) {
    if (n == 0) return;
    k_rays_from_user<<<(n + 255) / 256, 256, 0, st>>>(rays, skip, n, ray_o, ray_d);
    lc.n++;
}

SceneDev scene_entry(const DevScene& s, bool bvh8) {
    SceneDev e;
    e.nodes2 = s.nodes2;
    e.nodes8 = s.nodes8;
    e.tris = bvh8 ? s.tris8 : s.tris;
    e.mats = s.mats;
    for (int k = 0; k < 3; ++k) {
        e.env[k] = s.env[k];
        e.lo[k] = s.lo[k];
        e.hi[k] = s.hi[k];
    }
    e.env[3] = e.lo[3] = e.hi[3] = 0.0f;
    e.light_cdf = s.light_cdf;
    e.lights = s.lights;
    e.n_lights = s.n_lights;
    e.light_total = s.light_total;
    return e;
}

void launch_trace(const TraceArgs& a, cudaStream_t st, LaunchCount& lc) {
    if (a.n_max == 0) return;
    const int block = a.block;
    const size_t smem = (size_t)kSmemStack * block * sizeof(uint32_t);
    const size_t smem128 = (size_t)kSmemStack * 128 * sizeof(uint32_t);
    if (a.any_hit) { // visibility queries (cr_trace_rays with CR_OPT_ANY_HIT)
        const uint32_t grid = (a.n_max + block - 1) / block;
        if (a.bvh8)
            k_trace_bvh8<false, true><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                                 a.queue_count, a.n_max, a.hit, nullptr);
        else
            k_trace_bvh2<false, true><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                                 a.queue_count, a.n_max, a.hit, nullptr);
        lc.n++;
        return;
    }
    if (a.bvh8) {
        const uint32_t grid = (a.n_max + block - 1) / block;
        if (a.counters)
            k_trace_bvh8<true><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                          a.queue_count, a.n_max, a.hit, a.counters);
        else
            k_trace_bvh8<false><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                           a.queue_count, a.n_max, a.hit, nullptr);
        lc.n++;
        return;
    }
    if (a.two_phase && !a.counters && a.phase.state && a.queue && a.queue_count) {
        const uint32_t grid = (a.n_max + block - 1) / block;
        const uint32_t nb = (a.n_max + 255) / 256;
        k_trace_bvh2_phase<<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue, a.queue_count,
                                                      a.n_max, a.hit, a.phase.state, a.phase.susp, a.phase.budget, 0);
        k_susp_count<<<nb, 256, 0, st>>>(a.phase.susp, a.queue_count, a.n_max, a.phase.block_counts);
        launch_scan_counts(a.phase.block_counts, nb, a.phase.count2, st);
        k_susp_scatter<<<nb, 256, 0, st>>>(a.phase.susp, a.queue, a.queue_count, a.n_max, a.phase.block_counts,
                                          a.phase.queue2);
        k_trace_bvh2_phase<<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.phase.queue2,
                                                      a.phase.count2, a.n_max, a.hit, a.phase.state, nullptr,
                                                      0xffffffffu, 1);
        lc.n += 5;
        return;
    }
    if (a.packet && !a.counters) {
        const uint32_t grid = (a.n_max + block - 1) / block;
        k_trace_bvh2_packet<<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                       a.queue_count, a.n_max, a.hit);
        lc.n++;
        return;
    }
    if (a.speculative && !a.counters) {
        const uint32_t grid = (a.n_max + block - 1) / block;
        k_trace_bvh2_spec<<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue, a.queue_count,
                                                     a.n_max, a.hit);
        lc.n++;
        return;
    }
    if (a.persistent && !a.counters) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_bvh2_dynamic, 128, smem128);
        const uint32_t grid_max = (uint32_t)sms * (uint32_t)(per_sm > 0 ? per_sm : 1);
        const uint32_t need = (a.n_max + 127) / 128;
        k_trace_bvh2_dynamic<<<need < grid_max ? need : grid_max, 128, smem128, st>>>(
            a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue, a.queue_count, a.n_max, a.hit, a.work_counter,
            a.refill == 0 ? 8u : (a.refill > 32u ? 32u : a.refill));
    } else {
        const uint32_t grid = (a.n_max + block - 1) / block;
        if (a.counters)
            k_trace_bvh2<true><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                          a.queue_count, a.n_max, a.hit, a.counters);
        else
            k_trace_bvh2<false><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                           a.queue_count, a.n_max, a.hit, nullptr);
    }
    lc.n++;
}

void launch_hits_to_user(const float4* tris, const int2* hit, uint32_t n, int32_t* prim, float* t, cudaStream_t st,
                         LaunchCount& lc) {
    if (n == 0) return;
    k_hits_to_user<<<(n + 255) / 256, 256, 0, st>>>(tris, hit, n, prim, t);
    lc.n++;
}

} // namespace cr
