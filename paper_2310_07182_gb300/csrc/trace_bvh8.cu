// trace_bvh8.cu -- closest-hit and any-hit traversal of the BVH8-Q (8-wide nodes whose
// child boxes are quantised to 8 bits, after Ylitie, Karras and Laine 2017).  Same
// primitives and closest-hit rule as the BVH2 kernels (trace_common.cuh), so both layouts
// return the same hit bit for bit.
#include <cuda_runtime.h>

#include "cr_internal.h"
#include "trace_common.cuh"

namespace cr {
namespace {

// ------------------------------------------------------------------------------------
// BVH8-Q traversal with hit-mask node groups (the scheme of Ylitie, Karras and Laine 2017).
// Node layout (80 bytes, five 16-byte loads): w0 = origin xyz | exponent bytes + inner mask,
// w1 = first inner child, first triangle, 8 meta bytes, w2..w4 = the children's 8-bit
// low / high planes per axis.  Children sit in slots by the octant of their centroid, so
// visiting slot i ^ octant(d) for i = 0..7 goes roughly near to far without sorting.
//
// One iteration intersects one node: the 8 children are slab-tested straight from their
// bytes (one FMA per plane, with error bounds that keep the test conservative); hit inner
// children form a bit mask in visiting order, hit leaves a mask of their triangles, which
// are tested at once.  The nearest inner child is visited next and the rest of the mask is
// pushed as one (first child, mask) entry, so the stack holds at most one entry per tree
// level.  Inner children are stored in slot order: the child in slot s is first child +
// popc(inner mask below s).
constexpr int kStack8 = (int)kBvh8StackCapacity; // >= the tree depth (checked at scene creation)

// bytes of an 8-byte field (lo = slots 0..3, hi = slots 4..7) reordered so that byte i is
// slot i ^ oct
__device__ __forceinline__ void octant_order(uint32_t& lo, uint32_t& hi, uint32_t oct, uint32_t sel) {
    if (oct & 4u) {
        const uint32_t t = lo;
        lo = hi;
        hi = t;
    }
    lo = __byte_perm(lo, 0u, sel);
    hi = __byte_perm(hi, 0u, sel);
}

// byte i of the 8-byte field (lo, hi) as a float (exact)
template <int i>
__device__ __forceinline__ float qbyte(uint32_t lo, uint32_t hi) {
    return __uint2float_rn(((i < 4 ? lo : hi) >> (8 * (i & 3))) & 0xffu);
}

template <bool kCount, bool kAny = false>
__device__ __forceinline__ int2 trace_bvh8_one(const uint4* __restrict__ nodes, const float4* __restrict__ tris,
                                               float4 ro, float4 rd, unsigned long long& n_node,
                                               unsigned long long& n_tri, const SceneDev* dsc = nullptr) {
    const RayPre r = prep_ray(ro, rd);
    const int skip = __float_as_int(ro.w);
    const uint32_t oct = (rd.x < 0.0f ? 1u : 0u) | (rd.y < 0.0f ? 2u : 0u) | (rd.z < 0.0f ? 4u : 0u);
    const uint32_t o3 = oct & 3u;
    const uint32_t sel = o3 | ((1u ^ o3) << 4) | ((2u ^ o3) << 8) | ((3u ^ o3) << 12);
    Best best{rd.w, -1, 0x7fffffff};
    uint2 stack[kStack8];
    int sp = 0;
    uint32_t node = 0;
    while (true) {
        if (kCount) ++n_node;
        CR_DBG(if (!dbg_in_range(dsc, (uint32_t)node, kDbgNode, dsc->n_nodes)) break;)
        const uint4 w0 = __ldg(&nodes[5 * node + 0]);
        const uint4 w1 = __ldg(&nodes[5 * node + 1]);
        const uint4 w2 = __ldg(&nodes[5 * node + 2]);
        const uint4 w3 = __ldg(&nodes[5 * node + 3]);
        const uint4 w4 = __ldg(&nodes[5 * node + 4]);
        const float ox = __uint_as_float(w0.x), oy = __uint_as_float(w0.y), oz = __uint_as_float(w0.z);
        const float sx = __uint_as_float((w0.w & 0xffu) << 23);
        const float sy = __uint_as_float(((w0.w >> 8) & 0xffu) << 23);
        const float sz = __uint_as_float(((w0.w >> 16) & 0xffu) << 23);
        const uint32_t imask = w0.w >> 24;
        const uint32_t child_base = w1.x, tri_base = w1.y;
        uint32_t m_lo = w1.z, m_hi = w1.w;
        uint32_t lx_lo = w2.x, lx_hi = w2.y, ly_lo = w2.z, ly_hi = w2.w, lz_lo = w3.x, lz_hi = w3.y;
        uint32_t hx_lo = w3.z, hx_hi = w3.w, hy_lo = w4.x, hy_hi = w4.y, hz_lo = w4.z, hz_hi = w4.w;
        octant_order(m_lo, m_hi, oct, sel);
        octant_order(lx_lo, lx_hi, oct, sel);
        octant_order(ly_lo, ly_hi, oct, sel);
        octant_order(lz_lo, lz_hi, oct, sel);
        octant_order(hx_lo, hx_hi, oct, sel);
        octant_order(hy_lo, hy_hi, oct, sel);
        octant_order(hz_lo, hz_hi, oct, sel);
        const float tcull = __fmul_rn(best.t, kCullWiden);
        // Plane distances straight from the bytes: a plane at origin + q * step meets the ray
        // at fma(q, a, b) with a = step / d (exact, step is a power of two) and
        // b = (origin - o) / d.  Against the decoded plane fl(origin + q * step), whose box
        // the builder makes contain the child, this is off by at most a relative 2^-23 plus
        // 2^-23 |1/d| (|origin| + 255 step + |origin - o|); b is biased by twice that, down
        // for the entry plane and up for the exit plane, and the exit widened as in the
        // BVH2 test, so no child box the decoded form would enter is rejected (2^-100 more
        // covers a step / d that falls into the subnormal range).
        float ax, ay, az, blx, bhx, bly, bhy, blz, bhz;
        {
            const float dx = __fsub_rn(ox, r.ox), dy = __fsub_rn(oy, r.oy), dz = __fsub_rn(oz, r.oz);
            ax = __fmul_rn(sx, r.ix);
            ay = __fmul_rn(sy, r.iy);
            az = __fmul_rn(sz, r.iz);
            const float bx = __fmul_rn(dx, r.ix), by = __fmul_rn(dy, r.iy), bz = __fmul_rn(dz, r.iz);
            const float ex = __fmul_rn(__fmul_rn(__fadd_rn(__fadd_rn(fabsf(ox), __fmul_rn(255.0f, sx)), fabsf(dx)),
                                                 fabsf(r.ix)), 0x1.0p-22f) + 0x1.0p-100f;
            const float ey = __fmul_rn(__fmul_rn(__fadd_rn(__fadd_rn(fabsf(oy), __fmul_rn(255.0f, sy)), fabsf(dy)),
                                                 fabsf(r.iy)), 0x1.0p-22f) + 0x1.0p-100f;
            const float ez = __fmul_rn(__fmul_rn(__fadd_rn(__fadd_rn(fabsf(oz), __fmul_rn(255.0f, sz)), fabsf(dz)),
                                                 fabsf(r.iz)), 0x1.0p-22f) + 0x1.0p-100f;
            // the low plane is the entry one where 1/d >= 0
            blx = r.ix >= 0.0f ? __fsub_rn(bx, ex) : __fadd_rn(bx, ex);
            bhx = r.ix >= 0.0f ? __fadd_rn(bx, ex) : __fsub_rn(bx, ex);
            bly = r.iy >= 0.0f ? __fsub_rn(by, ey) : __fadd_rn(by, ey);
            bhy = r.iy >= 0.0f ? __fadd_rn(by, ey) : __fsub_rn(by, ey);
            blz = r.iz >= 0.0f ? __fsub_rn(bz, ez) : __fadd_rn(bz, ez);
            bhz = r.iz >= 0.0f ? __fadd_rn(bz, ez) : __fsub_rn(bz, ez);
        }
        uint32_t hits = 0, trimask = 0;
#define CR_BVH8_CHILD(i)                                                                                  \
    {                                                                                                     \
        const uint32_t meta = ((i < 4 ? m_lo : m_hi) >> (8 * (i & 3))) & 0xffu;                         \
        const bool inner = (imask >> ((uint32_t)(i) ^ oct)) & 1u;                                         \
        if (inner || meta >= 32u) {                                                                       \
            const float tlx = fmaf(qbyte<i>(lx_lo, lx_hi), ax, blx);                                      \
            const float thx = fmaf(qbyte<i>(hx_lo, hx_hi), ax, bhx);                                      \
            const float tly = fmaf(qbyte<i>(ly_lo, ly_hi), ay, bly);                                      \
            const float thy = fmaf(qbyte<i>(hy_lo, hy_hi), ay, bhy);                                      \
            const float tlz = fmaf(qbyte<i>(lz_lo, lz_hi), az, blz);                                      \
            const float thz = fmaf(qbyte<i>(hz_lo, hz_hi), az, bhz);                                      \
            const float tn = max3f(fminf(tlx, thx), fminf(tly, thy), fmaxf(fminf(tlz, thz), 0.0f));       \
            const float tf = min3f(fmaxf(tlx, thx), fmaxf(tly, thy), fmaxf(tlz, thz));                    \
            if (tn <= __fmul_rn(tf, kFarWiden) && tn <= tcull) {                                          \
                if (inner) hits |= 1u << (i);                                                             \
                else trimask |= ((1u << (meta >> 5)) - 1u) << (meta & 31u);                               \
            }                                                                                             \
        }                                                                                                 \
    }
        CR_BVH8_CHILD(0)
        CR_BVH8_CHILD(1)
        CR_BVH8_CHILD(2)
        CR_BVH8_CHILD(3)
        CR_BVH8_CHILD(4)
        CR_BVH8_CHILD(5)
        CR_BVH8_CHILD(6)
        CR_BVH8_CHILD(7)
#undef CR_BVH8_CHILD
        // the hit leaves' triangles
        while (trimask) {
            const uint32_t j = (uint32_t)__ffs(trimask) - 1u;
            trimask &= trimask - 1u;
            CR_DBG(if (!dbg_in_range(dsc, tri_base + j, kDbgTri, dsc->n_tris)) break;)
            test_leaf(tris, r, skip, tri_base + j, 1u, best, n_tri);
        }
        if (kAny && best.leaf >= 0) break;
        // next node: the nearest hit inner child of this node, else the next of a pushed group
        uint32_t base = child_base, im = imask;
        if (!hits) {
            if (sp == 0) break;
            --sp;
            base = stack[sp].x;
            hits = stack[sp].y & 0xffu;
            im = stack[sp].y >> 8;
        }
        const uint32_t i = (uint32_t)__ffs(hits) - 1u;
        hits &= hits - 1u;
        const uint32_t slot = i ^ oct;
        node = base + __popc(im & ((1u << slot) - 1u));
        if (hits) {
            stack[sp] = make_uint2(base, hits | (im << 8));
            sp = sp < kStack8 - 1 ? sp + 1 : sp; // scene creation checks depth < kStack8
        }
    }
    return make_int2(best.leaf, __float_as_int(best.t));
}

#ifndef CR_BVH8_MIN_BLOCKS
#define CR_BVH8_MIN_BLOCKS 8 // resident 128-thread blocks per SM the register budget is sized for
#endif

template <bool kCount, bool kAny = false>
__global__ void __launch_bounds__(128, CR_BVH8_MIN_BLOCKS) k_trace_bvh8(const SceneDev* __restrict__ scenes,
                             const uint16_t* __restrict__ slot_scene,
                             const float4* __restrict__ ray_o, const float4* __restrict__ ray_d,
                             const int32_t* __restrict__ queue, const uint32_t* __restrict__ queue_count,
                             uint32_t n_max, int2* __restrict__ hit, unsigned long long* counters) {
    const uint32_t n = queue_count ? min(*queue_count, n_max) : n_max;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long n_node = 0, n_tri = 0;
    if (i < n) {
        const int slot = queue ? queue[i] : (int)i;
        const SceneDev& sc = scenes[slot_scene ? slot_scene[slot] : 0];
        const float4 ro = ray_o[slot];
        const float4 rd = ray_d[slot];
        int2 h = make_int2(-1, __float_as_int(INFINITY));
        if (rd.w >= 0.0f) h = trace_bvh8_one<kCount, kAny>(sc.nodes8, sc.tris, ro, rd, n_node, n_tri, &sc);
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

// Shadow rays of next-event estimation over the BVH8-Q, one thread per position of the last shade's group
// queue (so a reuse group's rays run in adjacent lanes, as they were shaded).  A ray whose
// direction record has w = tmax > 0 is traced for visibility only; if nothing blocks it, its
// contribution is added to the path radiance of its slot.  Rays traced are counted.
__global__ void __launch_bounds__(128, CR_BVH8_MIN_BLOCKS) k_trace_shadow8(
    const SceneDev* __restrict__ scenes, const uint16_t* __restrict__ slot_scene, const float4* __restrict__ sh_o,
    const float4* __restrict__ sh_d, const float4* __restrict__ sh_c, const int32_t* __restrict__ group_queue,
    const uint32_t* __restrict__ group_count, uint32_t n_groups_max, uint32_t K, float4* __restrict__ radiance,
    unsigned long long* __restrict__ n_traced) {
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
            const int2 h = trace_bvh8_one<false, true>(sc.nodes8, sc.tris, ro, rd, dn, dt, &sc);
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


} // namespace

void launch_trace_bvh8(const TraceArgs& a, cudaStream_t st, LaunchCount& lc) {
    const int block = a.block;
    const size_t smem = 0;
    const uint32_t grid = (a.n_max + block - 1) / block;
    if (a.any_hit)
        k_trace_bvh8<false, true><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                             a.queue_count, a.n_max, a.hit, nullptr);
    else if (a.counters)
        k_trace_bvh8<true><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                      a.queue_count, a.n_max, a.hit, a.counters);
    else
        k_trace_bvh8<false><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                       a.queue_count, a.n_max, a.hit, nullptr);
    lc.n++;
}

void launch_shadow_rays_bvh8(const SceneDev* scenes, const uint16_t* slot_scene, const float4* sh_o,
                             const float4* sh_d, const float4* sh_c, const int32_t* group_queue,
                             const uint32_t* group_count, uint32_t n_groups_max, uint32_t K, float4* radiance,
                             unsigned long long* n_traced, cudaStream_t st, LaunchCount& lc) {
    const int block = 128;
    const size_t smem = 0;
    const uint32_t grid = (n_groups_max * K + block - 1) / block;
    k_trace_shadow8<<<grid, block, smem, st>>>(scenes, slot_scene, sh_o, sh_d, sh_c, group_queue, group_count,
                                               n_groups_max, K, radiance, n_traced);
    lc.n++;
}

} // namespace cr
