// trace_bvh4.cu -- closest-hit traversal of the BVH4 (4-wide nodes with FP32 child boxes,
// collapsed from the BVH2 in bvh4_build.cpp), one ray per thread.
//
// A node visit loads the node's seven 16-byte words (the near and far plane words of each
// axis picked by the ray's direction signs), tests the four child boxes with the BVH2
// kernel's conservative slab test (unused slots have NaN planes and never pass), and
// orders the hit children by entry distance: the distance bits with the child slot in the
// two low bits, sorted by a five-exchange network (the slot bits only reorder children whose
// distances agree to 21 bits, which changes the visit order, never the closest hit).  The
// nearest hit child is visited next; the others are pushed farthest first as (node, slot),
// on the BVH2 kernel's stack (shared memory, then a local array), and a pop reads the
// child's link from the node (cheaper than selecting every pushed child's link at once).
// Leaves are BVH2 leaves over the same triangle records, tested with the same watertight test
// and closest-hit rule, so the hits equal the BVH2 traversal's.
#include <cuda_runtime.h>

#include "cr_internal.h"
#include "trace_common.cuh"

namespace cr {
namespace {

#ifndef CR_TRACE4_MAXNREG
#define CR_TRACE4_MAXNREG 64
#endif

// The slab test of box_hit_fma with the near and far planes chosen by the ray: three min /
// max operations per box instead of nine.  Unused slots (NaN planes) still miss: the exit
// distance is NaN and the comparison fails.
__device__ __forceinline__ bool box_hit_nf(const RayPre& r, float nx, float fx, float ny, float fy, float nz, float fz,
                                           float onx, float ofx, float ony, float ofy, float onz, float ofz, float tcull,
                                           float& tn) {
    tn = fmaxf(max3f(fmaf(nx, r.ix, onx), fmaf(ny, r.iy, ony), fmaf(nz, r.iz, onz)), 0.0f);
    const float tf = min3f(fmaf(fx, r.ix, ofx), fmaf(fy, r.iy, ofy), fmaf(fz, r.iz, ofz));
    return tn <= __fmul_rn(tf, kFarWiden) && tn <= tcull;
}

__device__ __forceinline__ void sort2(uint32_t& a, uint32_t& b) {
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Pop a pushed (node, slot) entry and read that child's link from the node.
#define POP_CHILD(v)                                                                                  \
    do {                                                                                              \
        int e_;                                                                                       \
        STACK_POP_TOP(e_);                                                                            \
        (v) = __ldg(reinterpret_cast<const int*>(nodes + 8 * (size_t)(e_ >> 2) + 6) + (e_ & 3));      \
    } while (0)

// dsc: the scene-table entry, read only by the index checks of a debug build.
template <bool kCount>
__device__ __forceinline__ int2 trace_bvh4_one(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                               float4 ro, float4 rd, uint32_t* sstack, unsigned long long& n_node,
                                               unsigned long long& n_tri, const SceneDev* dsc = nullptr) {
    constexpr int kSmemS = kSmemStack;
    const RayPre r = prep_ray(ro, rd);
    const int skip = __float_as_int(ro.w);
    Best best{rd.w, -1, 0x7fffffff};
    int lstack[kBvh4StackCapacity - kSmemS];
    const int stride = blockDim.x;
    int sp = 0;
    int node = 0;
    float tcull = __fmul_rn(best.t, kCullWiden);
    uint32_t* top = sstack;
    // the near and far plane of each axis follow from the sign of 1/d (the offsets are biased
    // by that sign too, so this equals the min / max of the two plane distances): their word
    // offsets in the node and their distance offsets, once per ray
    const int sxn = r.ix < 0.0f, syn = r.iy < 0.0f, szn = r.iz < 0.0f;
    const int wnx = sxn, wfx = 1 - sxn, wny = 2 + syn, wfy = 3 - syn, wnz = 4 + szn, wfz = 5 - szn;
    const float onx = sxn ? r.hix : r.lox, ofx = sxn ? r.lox : r.hix;
    const float ony = syn ? r.hiy : r.loy, ofy = syn ? r.loy : r.hiy;
    const float onz = szn ? r.hiz : r.loz, ofz = szn ? r.loz : r.hiz;
    while (true) {
        while (node >= 0) {
            if (kCount) ++n_node;
            CR_DBG(if (!dbg_in_range(dsc, (uint32_t)node, kDbgNode, dsc->n_nodes4)) {
                node = 0x7fffffff;
                break;
            })
            const float4* q = nodes + 8 * (size_t)node;
            const float4 nx = __ldg(q + wnx), fx = __ldg(q + wfx), ny = __ldg(q + wny), fy = __ldg(q + wfy);
            const float4 nz = __ldg(q + wnz), fz = __ldg(q + wfz), cc = __ldg(q + 6);
            const int c0 = __float_as_int(cc.x), c1 = __float_as_int(cc.y), c2 = __float_as_int(cc.z),
                      c3 = __float_as_int(cc.w);
            float t0, t1, t2, t3;
            const bool h0 = box_hit_nf(r, nx.x, fx.x, ny.x, fy.x, nz.x, fz.x, onx, ofx, ony, ofy, onz, ofz, tcull, t0);
            const bool h1 = box_hit_nf(r, nx.y, fx.y, ny.y, fy.y, nz.y, fz.y, onx, ofx, ony, ofy, onz, ofz, tcull, t1);
            const bool h2 = box_hit_nf(r, nx.z, fx.z, ny.z, fy.z, nz.z, fz.z, onx, ofx, ony, ofy, onz, ofz, tcull, t2);
            const bool h3 = box_hit_nf(r, nx.w, fx.w, ny.w, fy.w, nz.w, fz.w, onx, ofx, ony, ofy, onz, ofz, tcull, t3);
            // entry distances are >= 0, so their bits order like the floats; misses sort last
            uint32_t k0 = h0 ? (__float_as_uint(t0) & ~3u) : 0xffffffffu;
            uint32_t k1 = h1 ? ((__float_as_uint(t1) & ~3u) | 1u) : 0xffffffffu;
            uint32_t k2 = h2 ? ((__float_as_uint(t2) & ~3u) | 2u) : 0xffffffffu;
            uint32_t k3 = h3 ? ((__float_as_uint(t3) & ~3u) | 3u) : 0xffffffffu;
            const int nh = (int)h0 + (int)h1 + (int)h2 + (int)h3;
            if (nh == 0) {
                if (sp == 0) {
                    node = 0x7fffffff;
                    break;
                }
                POP_CHILD(node);
                continue;
            }
            sort2(k0, k1);
            sort2(k2, k3);
            sort2(k0, k2);
            sort2(k1, k3);
            sort2(k1, k2);
            const auto link = [&](uint32_t k) {
                const uint32_t s = k & 3u;
                return s == 0u ? c0 : s == 1u ? c1 : s == 2u ? c2 : c3;
            };
            const int ent = node << 2;
            if (nh == 4) STACK_PUSH_TOP(ent | (int)(k3 & 3u));
            if (nh >= 3) STACK_PUSH_TOP(ent | (int)(k2 & 3u));
            if (nh >= 2) STACK_PUSH_TOP(ent | (int)(k1 & 3u));
            node = link(k0);
        }
        if (node == 0x7fffffff) break;
        // leaf: a BVH2 leaf code
        const uint32_t code = (uint32_t)(~node);
        CR_DBG(if (!dbg_in_range(dsc, (code >> 2) + (code & 3u), kDbgTri, dsc->n_tris)) break;)
        test_leaf(tris, r, skip, code >> 2, (code & 3u) + 1u, best, n_tri);
        tcull = __fmul_rn(best.t, kCullWiden);
        if (sp == 0) break;
        POP_CHILD(node);
    }
    return make_int2(best.leaf, __float_as_int(best.t));
}

template <bool kCount>
__global__ void __maxnreg__(CR_TRACE4_MAXNREG) k_trace_bvh4(const SceneDev* __restrict__ scenes,
                                                             const uint16_t* __restrict__ slot_scene,
                                                             const float4* __restrict__ ray_o,
                                                             const float4* __restrict__ ray_d,
                                                             const int32_t* __restrict__ queue,
                                                             const uint32_t* __restrict__ queue_count, uint32_t n_max,
                                                             int2* __restrict__ hit, unsigned long long* counters) {
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
            h = trace_bvh4_one<kCount>(sc.nodes4, sc.tris, ro, rd, smem_stack + threadIdx.x, n_node, n_tri, &sc);
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

} // namespace

// Closest hits of the queued rays through the BVH4 (the scene entries' nodes4 and tris).
void launch_trace_bvh4(const TraceArgs& a, cudaStream_t st, LaunchCount& lc) {
    if (a.n_max == 0) return;
    const int block = a.block;
    const uint32_t grid = (a.n_max + block - 1) / block;
    const size_t smem = (size_t)block * kSmemStack * sizeof(uint32_t);
    if (a.counters)
        k_trace_bvh4<true><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue, a.queue_count,
                                                       a.n_max, a.hit, a.counters);
    else
        k_trace_bvh4<false><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                        a.queue_count, a.n_max, a.hit, nullptr);
    lc.n++;
}

} // namespace cr
