// trace.cu -- closest-hit BVH2 traversal (the intersection step, which dominates path
// tracing time, Sec. 1), one ray per thread.
//
// Stackful while-while traversal of the 64-byte two-child nodes: both child boxes are
// fetched with four 16-byte read-only loads, tested with a conservative slab test, the
// nearer hit child is visited first and the farther one pushed.  The traversal stack lives
// in shared memory (kSmemStack entries per thread, interleaved so that a warp's pushes hit
// distinct banks) and continues in a per-thread local array for deeper trees.  Leaves hold
// up to four triangles tested with the watertight test of Woop, Benthin and Wald (2013).
// The primitives and the closest-hit rule shared with the BVH8-Q kernels (trace_bvh8.cu)
// are in trace_common.cuh.
#include <cuda_runtime.h>

#include "cr_internal.h"
#include "trace_common.cuh"

namespace cr {
namespace {


// kAny: visibility only; the traversal ends at the first triangle hit before the ray's tmax.
// kSmemS: stack entries per thread kept in shared memory (8, 16 or 32; deeper ones go to a
// local array), a launch-shape knob of the autotuner.
// dsc: the scene-table entry, read only by the index checks of a debug build.
template <bool kCount, bool kAny = false, int kSmemS = kSmemStack>
__device__ __forceinline__ int2 trace_bvh2_one(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                               float4 ro, float4 rd, uint32_t* sstack, unsigned long long& n_node,
                                               unsigned long long& n_tri, const SceneDev* dsc = nullptr) {
    const RayPre r = prep_ray(ro, rd);
    const int skip = __float_as_int(ro.w);
    Best best{rd.w, -1, 0x7fffffff};
    int lstack[kStackTotal - kSmemS];
    const int stride = blockDim.x;
    int sp = 0;
    int node = 0;
    float tcull = __fmul_rn(best.t, kCullWiden); // changes only after a leaf
    uint32_t* top = sstack; // next free shared-memory stack entry (stays at the end once full)
    while (true) {
        while (node >= 0) {
            if (kCount) ++n_node;
            CR_DBG(if (!dbg_in_range(dsc, (uint32_t)node, kDbgNode, dsc->n_nodes)) {
                node = 0x7fffffff;
                break;
            })
            const float4 n0 = __ldg(&nodes[4 * node + 0]);
            const float4 n1 = __ldg(&nodes[4 * node + 1]);
            const float4 n2 = __ldg(&nodes[4 * node + 2]);
            const float4 n3 = __ldg(&nodes[4 * node + 3]);
            float t0, t1;
            const bool h0 = box_hit_fma(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tcull, t0);
            const bool h1 = box_hit_fma(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tcull, t1);
            const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            if (h0 && h1) {
                const bool first0 = t0 <= t1;
                const int near = first0 ? c0 : c1, far = first0 ? c1 : c0;
                STACK_PUSH_TOP(far);
                node = near;
            } else if (h0 || h1) {
                node = h0 ? c0 : c1;
            } else {
                if (sp == 0) { node = 0x7fffffff; break; }
                STACK_POP_TOP(node);
            }
        }
        if (node == 0x7fffffff) break;
        // leaf
        const uint32_t code = (uint32_t)(~node);
        CR_DBG(if (!dbg_in_range(dsc, (code >> 2) + (code & 3u), kDbgTri, dsc->n_tris)) break;)
        test_leaf(tris, r, skip, code >> 2, (code & 3u) + 1u, best, n_tri);
        if (kAny && best.leaf >= 0) break;
        tcull = __fmul_rn(best.t, kCullWiden);
        if (sp == 0) break;
        STACK_POP_TOP(node);
    }
    return make_int2(best.leaf, __float_as_int(best.t));
}

#ifndef CR_TRACE_MAXNREG
#define CR_TRACE_MAXNREG 48 // 42 warps resident per SM (10 blocks of 128 or 21 of 64 threads); 40 spills
#endif

template <bool kCount, bool kAny = false, int kSmemS = kSmemStack>
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
            h = trace_bvh2_one<kCount, kAny, kSmemS>(sc.nodes2, sc.tris, ro, rd, smem_stack + threadIdx.x, n_node,
                                                     n_tri, &sc);
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
    constexpr int kSmemS = kSmemStack;
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
    constexpr int kSmemS = kSmemStack;
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

// Shadow rays of next-event estimation, one thread per position of the last shade's group
// queue (so a reuse group's rays run in adjacent lanes, as they were shaded).  A ray whose
// direction record has w = tmax > 0 is traced for visibility only; if nothing blocks it, its
// contribution is added to the path radiance of its slot.  Rays traced are counted.
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
            const int2 h = trace_bvh2_one<false, true>(sc.nodes2, sc.tris, ro, rd, smem_stack + threadIdx.x, dn, dt, &sc);
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
    if (bvh8) {
        launch_shadow_rays_bvh8(scenes, slot_scene, sh_o, sh_d, sh_c, group_queue, group_count, n_groups_max, K,
                                radiance, n_traced, st, lc);
        return;
    }
    k_trace_shadow<<<grid, block, smem, st>>>(scenes, slot_scene, sh_o, sh_d, sh_c, group_queue, group_count,
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
    e.nodes4 = s.nodes4;
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
    e.n_nodes = bvh8 ? s.n_nodes8 : s.n_nodes2;
    e.n_tris = s.n_tri;
    e.n_mats = s.n_mat;
    e.err = s.err;
    return e;
}

void launch_trace(const TraceArgs& a, cudaStream_t st, LaunchCount& lc) {
    if (a.n_max == 0) return;
    const int block = a.block;
    const size_t smem = (size_t)kSmemStack * block * sizeof(uint32_t);
    const size_t smem128 = (size_t)kSmemStack * 128 * sizeof(uint32_t);
    if (a.bvh8) { // BVH8-Q kernels (trace_bvh8.cu)
        launch_trace_bvh8(a, st, lc);
        return;
    }
    if (a.bvh4 && !a.any_hit) { // BVH4 kernel (trace_bvh4.cu)
        launch_trace_bvh4(a, st, lc);
        return;
    }
    if (a.any_hit) { // visibility queries (cr_trace_rays with CR_OPT_ANY_HIT)
        const uint32_t grid = (a.n_max + block - 1) / block;
        k_trace_bvh2<false, true><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
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
        if (a.counters) {
            k_trace_bvh2<true><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                          a.queue_count, a.n_max, a.hit, a.counters);
        } else if (a.stack == 8) {
            k_trace_bvh2<false, false, 8><<<grid, block, (size_t)8 * block * 4, st>>>(
                a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue, a.queue_count, a.n_max, a.hit, nullptr);
        } else if (a.stack == 32) {
            const size_t smem32 = (size_t)32 * block * 4;
            if (smem32 > 48 * 1024) // 512-thread blocks need the opt-in beyond 48 KB
                cudaFuncSetAttribute(k_trace_bvh2<false, false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem32);
            k_trace_bvh2<false, false, 32><<<grid, block, smem32, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d,
                                                                        a.queue, a.queue_count, a.n_max, a.hit,
                                                                        nullptr);
        } else {
            k_trace_bvh2<false><<<grid, block, smem, st>>>(a.scenes, a.slot_scene, a.ray_o, a.ray_d, a.queue,
                                                           a.queue_count, a.n_max, a.hit, nullptr);
        }
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
