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
// Closest-hit rule, identical for the BVH2 and BVH8-Q kernels: accept t > 0 if
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

template <bool kCount>
__device__ __forceinline__ int2 trace_bvh2_one(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                               float4 ro, float4 rd, uint32_t* sstack, unsigned long long& n_node,
                                               unsigned long long& n_tri) {
    const RayPre r = prep_ray(ro, rd);
    const int skip = __float_as_int(ro.w);
    Best best{rd.w, -1, 0x7fffffff};
    int lstack[kStackTotal - kSmemStack];
    int sp = 0;
    int node = 0;
    const int stride = blockDim.x;
    while (true) {
        while (node >= 0) {
            if (kCount) ++n_node;
            const float4 n0 = __ldg(&nodes[4 * node + 0]);
            const float4 n1 = __ldg(&nodes[4 * node + 1]);
            const float4 n2 = __ldg(&nodes[4 * node + 2]);
            const float4 n3 = __ldg(&nodes[4 * node + 3]);
            const float tcull = __fmul_rn(best.t, kCullWiden);
            const float t0 = box_entry(r, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, tcull);
            const float t1 = box_entry(r, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, tcull);
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
            } else {
                if (sp == 0) { node = 0x7fffffff; break; }
                --sp;
                node = sp < kSmemStack ? (int)sstack[sp * stride] : lstack[sp - kSmemStack];
            }
        }
        if (node == 0x7fffffff) break;
        // leaf
        const uint32_t code = (uint32_t)(~node);
        test_leaf(tris, r, skip, code >> 2, (code & 3u) + 1u, best, n_tri);
        if (sp == 0) break;
        --sp;
        node = sp < kSmemStack ? (int)sstack[sp * stride] : lstack[sp - kSmemStack];
    }
    return make_int2(best.leaf, __float_as_int(best.t));
}

template <bool kCount>
__global__ void k_trace_bvh2(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                             const float4* __restrict__ ray_o, const float4* __restrict__ ray_d,
                             const int32_t* __restrict__ queue, const uint32_t* __restrict__ queue_count,
                             uint32_t n_max, int2* __restrict__ hit, unsigned long long* counters) {
    extern __shared__ uint32_t smem_stack[];
    const uint32_t n = queue_count ? min(*queue_count, n_max) : n_max;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long n_node = 0, n_tri = 0;
    if (i < n) {
        const int slot = queue ? queue[i] : (int)i;
        const float4 ro = ray_o[slot];
        const float4 rd = ray_d[slot];
        int2 h = make_int2(-1, __float_as_int(INFINITY));
        if (rd.w >= 0.0f) h = trace_bvh2_one<kCount>(nodes, tris, ro, rd, smem_stack + threadIdx.x, n_node, n_tri);
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

// Persistent variant: a fixed grid of resident blocks; each warp takes 32 rays at a time
// from an atomic counter until the queue is exhausted.  The loop ends when the counter
// passes the ray count, which it must since every iteration advances it.
__global__ void k_trace_bvh2_persistent(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                        const float4* __restrict__ ray_o, const float4* __restrict__ ray_d,
                                        const int32_t* __restrict__ queue, const uint32_t* __restrict__ queue_count,
                                        uint32_t n_max, int2* __restrict__ hit, uint32_t* work) {
    extern __shared__ uint32_t smem_stack[];
    const uint32_t n = queue_count ? min(*queue_count, n_max) : n_max;
    const int lane = threadIdx.x & 31;
    unsigned long long dn = 0, dt = 0;
    while (true) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(work, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        const uint32_t i = base + lane;
        if (i < n) {
            const int slot = queue ? queue[i] : (int)i;
            const float4 ro = ray_o[slot];
            const float4 rd = ray_d[slot];
            int2 h = make_int2(-1, __float_as_int(INFINITY));
            if (rd.w >= 0.0f) h = trace_bvh2_one<false>(nodes, tris, ro, rd, smem_stack + threadIdx.x, dn, dt);
            hit[slot] = h;
        }
    }
}

__global__ void k_hits_to_user(const float4* __restrict__ tris, const int2* __restrict__ hit, uint32_t n,
                               int32_t* __restrict__ prim, float* __restrict__ t) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 h = hit[i];
    prim[i] = h.x >= 0 ? __float_as_int(__ldg(&tris[3 * h.x]).w) : -1;
    t[i] = __int_as_float(h.y);
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

void launch_rays_from_user(const float* rays, const int32_t* skip, uint32_t n, float4* ray_o, float4* ray_d,
                           cudaStream_t st, LaunchCount& lc) {
    if (n == 0) return;
    k_rays_from_user<<<(n + 255) / 256, 256, 0, st>>>(rays, skip, n, ray_o, ray_d);
    lc.n++;
}

void launch_trace(const DevScene& s, const TraceArgs& a, cudaStream_t st, LaunchCount& lc) {
    if (a.n_max == 0) return;
    const int block = a.block;
    const size_t smem = (size_t)kSmemStack * block * sizeof(uint32_t);
    if (a.persistent && !a.counters) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_bvh2_persistent, block, smem);
        const uint32_t grid_max = (uint32_t)sms * (uint32_t)(per_sm > 0 ? per_sm : 1);
        const uint32_t need = (a.n_max + block - 1) / block;
        k_trace_bvh2_persistent<<<need < grid_max ? need : grid_max, block, smem, st>>>(
            s.nodes2, s.tris, a.ray_o, a.ray_d, a.queue, a.queue_count, a.n_max, a.hit, a.work_counter);
    } else {
        const uint32_t grid = (a.n_max + block - 1) / block;
        if (a.counters)
            k_trace_bvh2<true><<<grid, block, smem, st>>>(s.nodes2, s.tris, a.ray_o, a.ray_d, a.queue, a.queue_count,
                                                          a.n_max, a.hit, a.counters);
        else
            k_trace_bvh2<false><<<grid, block, smem, st>>>(s.nodes2, s.tris, a.ray_o, a.ray_d, a.queue,
                                                           a.queue_count, a.n_max, a.hit, nullptr);
    }
    lc.n++;
}

void launch_hits_to_user(const DevScene& s, const int2* hit, uint32_t n, int32_t* prim, float* t, cudaStream_t st,
                         LaunchCount& lc) {
    if (n == 0) return;
    k_hits_to_user<<<(n + 255) / 256, 256, 0, st>>>(s.tris, hit, n, prim, t);
    lc.n++;
}

} // namespace cr
