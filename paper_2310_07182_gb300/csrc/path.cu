// path.cu -- wavefront path-tracing stages around the traversal: primary ray generation
// in reuse-group slot order, the fused shade / classify / reuse / spawn stage with the
// group-granular path compaction inside it (or, as an option, a separate order-preserving
// compaction), the Morton-sort comparator, and the accumulation that finishes a pass.
//
// Slot layout (Sec. 3.3): the image is cut into W x H tiles; inside tile t the pixel with
// row-major index i goes to slot t*m + sigma_{t,f}(i), where sigma is the tile's and
// frame's LCG shuffle.  Group g of the tile is slots [t*m + g*K, t*m + (g+1)*K), so a
// group's members are K adjacent lanes of one warp (K <= 32) or of one block (K <= 256).
#include <cuda_runtime.h>

#include "cr_internal.h"
#include "debug_checks.cuh"
#include "device_math.cuh"

namespace cr {
namespace {

using namespace dev;

// ------------------------------------------------------------------------------------
// Interleaved grouping (Sec. 3.3).  The tile's LCG x_{k+1} = (a x_k + c) mod m is
// evaluated at index i by composing the affine map with itself (binary powers), so each
// thread finds sigma(i) in log2(m) steps.
struct Lcg {
    uint32_t a, c, x0;
};

__device__ __forceinline__ Lcg tile_lcg(uint64_t seed, uint32_t tile, uint32_t frame, uint32_t m, uint32_t interleave) {
    if (!interleave) return Lcg{1u, 1u, 0u};
    const uint4 h = philox_seed(seed, tile, frame, kTagInterleave, 0u);
    const uint32_t q4 = m / 4 > 0 ? m / 4 : 1, q2 = m / 2 > 0 ? m / 2 : 1;
    return Lcg{4u * (h.x % q4) + 1u, 2u * (h.y % q2) + 1u, h.z % m};
}

__device__ __forceinline__ uint32_t sigma_of(const Lcg& L, uint32_t i, uint32_t m, uint32_t interleave) {
    if (!interleave) return i;
    const uint32_t mask = m - 1u;
    uint32_t A = 1u, C = 0u;           // accumulated map x -> A x + C
    uint32_t pa = L.a & mask, pc = L.c & mask; // current power of the step map
    for (uint32_t e = i; e; e >>= 1) {
        if (e & 1u) {
            A = (pa * A) & mask;
            C = (pa * C + pc) & mask;
        }
        const uint32_t na = (pa * pa) & mask;
        pc = (pa * pc + pc) & mask;
        pa = na;
    }
    return (A * L.x0 + C) & mask;
}

// Primary ray through (px + u, py + v): pinhole camera with a vertical field of view.
__device__ __forceinline__ V3 camera_dir(const CamBasis& c, uint32_t px, uint32_t py, float u, float v) {
    const float sx = fm(fs(fd(fm(2.0f, fa((float)px, u)), (float)c.width), 1.0f), c.tx);
    const float sy = fm(fs(1.0f, fd(fm(2.0f, fa((float)py, v)), (float)c.height)), c.ty);
    const V3 d = v3(fa(fa(c.fwd[0], fm(sx, c.right[0])), fm(sy, c.up[0])),
                    fa(fa(c.fwd[1], fm(sx, c.right[1])), fm(sy, c.up[1])),
                    fa(fa(c.fwd[2], fm(sx, c.right[2])), fm(sy, c.up[2])));
    return normalize3(d);
}

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    uint32_t x = v;
    for (uint32_t off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        const uint32_t nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? s_warp[lane] : 0u;
        for (uint32_t off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < nw) s_warp[lane] = s;
    }
    __syncthreads();
    const uint32_t nw = blockDim.x >> 5;
    total = s_warp[nw - 1];
    const uint32_t excl = x - v + (w > 0 ? s_warp[w - 1] : 0u);
    __syncthreads();
    return excl;
}

// Job of a pass tile: the last job whose first tile is <= tile (jobs are in tile order).
__device__ __forceinline__ uint32_t job_of_tile(const JobDev* jobs, uint32_t n_jobs, uint32_t tile) {
    uint32_t lo = 0, hi = n_jobs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (jobs[mid].tile_base <= tile) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Entry of a rolling launch list covering unit u (the last entry whose prefix is <= u).
__device__ __forceinline__ uint32_t launch_entry(const uint32_t* prefix, uint32_t n, uint32_t u) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One block covers blockDim / m whole tiles: every thread finds sigma of its pixel, the
// inverse map is built in shared memory, then thread j writes slot j of its tile so the
// slot arrays are written contiguously.
// primary_queue (optional): entry tile * m + i = the slot of the tile's i-th pixel, so that the
// primary trace can visit a tile's pixels in row-major order (compact pixel blocks per warp).
// Rolling wavefront: the launch covers the tiles of the jobs that start a sample (launch
// lists), their slots lie in each job's own slot range, and the block appends its live slots
// to the ray queue and its groups with a live member to the next group queue.
__global__ void k_raygen(PassArgs p, int32_t* __restrict__ pixel, uint16_t* __restrict__ slot_job,
                         uint16_t* __restrict__ slot_scene, float4* __restrict__ ray_o, float4* __restrict__ ray_d,
                         float4* __restrict__ beta, float4* __restrict__ radiance, uint8_t* __restrict__ alive,
                         int32_t* __restrict__ primary_queue, uint32_t* __restrict__ queue_counts) {
    extern __shared__ uint16_t inv[];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_base[2];
    // the shade kernels append to the per-bounce queue counters: zero them for this pass
    if (!p.rolling && blockIdx.x == 0 && threadIdx.x < kQueueCountWords) queue_counts[threadIdx.x] = 0;
    const uint32_t m = p.m;
    const uint32_t tiles_per_block = blockDim.x / m;
    const uint32_t tl = threadIdx.x / m, j = threadIdx.x % m;
    const uint32_t tile = blockIdx.x * tiles_per_block + tl;
    const bool in = tl < tiles_per_block && tile < p.n_tiles;
    uint32_t jid = 0, t = 0, slot_tile = tile;
    if (in) {
        if (p.rolling) {
            const uint32_t e = launch_entry(p.launch_prefix, p.n_launch, tile);
            jid = p.launch_job[e];
            t = tile - p.launch_prefix[e];
            slot_tile = p.jobs[jid].slot_tile + t;
        } else {
            jid = job_of_tile(p.jobs, p.n_jobs, tile);
            t = tile - p.jobs[jid].tile_base;
        }
        const JobDev& J = p.jobs[jid];
        const Lcg L = tile_lcg(J.seed, t + J.tile_first, J.frame, m, J.interleave);
        const uint32_t s = sigma_of(L, j, m, J.interleave);
        inv[tl * m + s] = (uint16_t)j;
        if (primary_queue && !p.rolling) primary_queue[tile * m + j] = (int32_t)(tile * m + s);
    }
    __syncthreads();
    bool live = false;
    uint32_t slot = 0;
    if (in) {
        const JobDev& J = p.jobs[jid];
        const uint32_t tt = t + J.tile_first;
        const uint32_t i = inv[tl * m + j];
        const uint32_t tx = tt % J.tiles_x, ty = tt / J.tiles_x;
        const uint32_t px = tx * p.tile_w + i % p.tile_w, py = ty * p.tile_h + i / p.tile_w;
        slot = slot_tile * m + j;
        slot_job[slot] = (uint16_t)jid;
        slot_scene[slot] = (uint16_t)J.scene;
        if (px < J.cam.width && py < J.cam.height) {
            const uint32_t pix = py * J.cam.width + px;
            const uint4 h = philox_seed(J.seed, pix, J.frame, 0u, kTagCamera);
            const V3 d = camera_dir(J.cam, px, py, unit24(h.x), unit24(h.y));
            pixel[slot] = (int32_t)pix;
            ray_o[slot] = make_float4(J.cam.pos[0], J.cam.pos[1], J.cam.pos[2], __int_as_float(-1));
            ray_d[slot] = make_float4(d.x, d.y, d.z, INFINITY);
            beta[slot] = make_float4(1.0f, 1.0f, 1.0f, 0.0f); // w: direction density, 0 for camera rays
            radiance[slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            alive[slot] = 1;
            live = true;
        } else {
            pixel[slot] = -1;
            ray_d[slot] = make_float4(0.0f, 0.0f, 0.0f, -1.0f);
            alive[slot] = 0;
        }
    }
    if (!p.rolling) return;
    // rolling: append the live slots (this iteration's trace) and the groups with a live member
    // (the next iteration's shade); a group is K consecutive slots, i.e. K consecutive threads
    uint32_t* grp_live = reinterpret_cast<uint32_t*>(inv + ((blockDim.x + 1) & ~1u));
    if (threadIdx.x < blockDim.x / p.k) grp_live[threadIdx.x] = 0u;
    __syncthreads();
    if (live) grp_live[threadIdx.x / p.k] = 1u;
    __syncthreads();
    const bool head = in && j % p.k == 0 && grp_live[threadIdx.x / p.k] != 0u;
    uint32_t tot_r, tot_g;
    const uint32_t rr = block_excl_scan(live ? 1u : 0u, s_warp, tot_r);
    const uint32_t rg = block_excl_scan(head ? 1u : 0u, s_warp, tot_g);
    if (threadIdx.x == 0) {
        s_base[0] = tot_r ? atomicAdd(&p.queue_counts[0], tot_r) : 0u;
        s_base[1] = tot_g ? atomicAdd(&p.queue_counts[1], tot_g) : 0u;
    }
    __syncthreads();
    if (live) p.ray_queue[s_base[0] + rr] = (int32_t)slot;
    if (head) p.group_queue_out[s_base[1] + rg] = (int32_t)(slot / p.k);
}

__global__ void k_groups(CamBasis cam, uint32_t tile_w, uint32_t tile_h, uint32_t interleave, uint64_t seed,
                         uint32_t frame, uint32_t* __restrict__ slot_of_pixel) {
    const uint32_t pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= cam.width * cam.height) return;
    const uint32_t m = tile_w * tile_h;
    const uint32_t tiles_x = (cam.width + tile_w - 1) / tile_w;
    const uint32_t px = pix % cam.width, py = pix / cam.width;
    const uint32_t tile = (py / tile_h) * tiles_x + px / tile_w;
    const uint32_t i = (py % tile_h) * tile_w + px % tile_w;
    const Lcg L = tile_lcg(seed, tile, frame, m, interleave);
    slot_of_pixel[pix] = tile * m + sigma_of(L, i, m, interleave);
}

// ------------------------------------------------------------------------------------
// Shade + classify + reuse + spawn (Sec. 3.2), one thread per slot of the alive groups.
struct ShadeArgs {
    const JobDev* jobs;
    const SceneDev* scenes;
    const uint16_t* slot_job;
    int32_t* pixel;
    float4* ray_o;
    float4* ray_d;
    const int2* hit;
    float4* beta;
    float4* radiance;
    uint8_t* alive;
    const int32_t* group_queue; // NULL: all groups in order
    const uint32_t* group_count;
    uint32_t n_groups_max;
    cr_debug dbg;
    uint32_t npx;
    // next-event estimation: shadow ray records per slot (NULL when no job uses it)
    float4* shadow_o;
    float4* shadow_d;
    float4* shadow_c;
    // queue compaction in the shade (ray_queue NULL: this launch does not compact)
    int32_t* ray_queue;              // continuing slots
    int32_t* group_queue_out;        // groups with a continuing member
    uint32_t* queue_counts;          // [0] rays, [1] groups appended (zeroed by raygen)
    unsigned long long* rays_queued; // running total of rays queued at this bounce
    uint32_t* queue_err;             // set if an append would overflow a queue (never expected)
    uint32_t ray_cap, group_cap;
};

struct Member {
    int pix;
    bool alive;
    bool final_pass; // the job's last secondary ray has been traced
    bool reuse;      // the job reuses directions at this bounce
    bool world;      // the job reuses world-space directions at this bounce (Sec. 3.1 ablation)
    bool nee;        // the job uses next-event estimation
    bool nee_shared; // ... with one light point per group
    bool hdonor;     // hybrid groups: diffuse members reuse the first diffuse member's sample
    bool cosgl;      // a GGX point in the diffuse class while reusing: cosine samples, pi f weights
    uint32_t scene;  // scene table index
    uint32_t type;   // material type of the shading point
    float rough;     // its roughness (the IOR of a dielectric)
    float hemi;      // +1: diffuse lobe in the upper hemisphere, -1: lower (translucent)
    bool front;      // the incoming ray met the triangle's front face
    uint64_t seed;
    uint32_t frame;
    uint32_t bounce; // this shading step's bounce (the launch's, or the job's own when rolling)
    int cls;
    V3 n, t, b, wo;
    float albedo[3];
    V3 wl;    // chosen tangent-space exit direction
    float w[3];
    bool valid;
    int orig;
};

// Shading point of a hit: geometric normal facing the incoming ray, tangent frame, wo.
// Weight pi f(wo, wi) (= f cos / p_cos) of a cosine-class GGX point for the tangent-space
// direction wl; usable when both it and wo lie above the surface.
__device__ __forceinline__ void rough_weight(Member& mb, V3 wl) {
    float f[3];
    eval_ggx(mb.wo, wl, mb.rough, mb.albedo, f);
    mb.w[0] = fm(3.14159265358979f, f[0]);
    mb.w[1] = fm(3.14159265358979f, f[1]);
    mb.w[2] = fm(3.14159265358979f, f[2]);
    mb.valid = wl.z > 0.0f && mb.wo.z > 0.0f;
}

// Radiance picked up where a ray ends without scattering.  Miss: beta times the constant
// environment.
__device__ __forceinline__ void add_environment(const SceneDev& sc, const float4 bt, float3& L) {
    L.x = fa(L.x, fm(bt.x, sc.env[0]));
    L.y = fa(L.y, fm(bt.y, sc.env[1]));
    L.z = fa(L.z, fm(bt.z, sc.env[2]));
}

// Emitter (triangle v0 v1 v2, emission m1.yzw): beta times the emission.  Under next-event
// estimation the emission met by a BSDF-sampled ray is weighed against the light sample that
// could have found it (power heuristic): the ray's direction had density beta.w (0: camera
// ray or mirror, full weight), a light sample density r^2 / (cos_l A).
__device__ __forceinline__ void add_emission(const SceneDev& sc, const float4 v0, const float4 v1, const float4 v2,
                                             const float4 m1, const float4 bt, const int2 h, const float4 d4,
                                             bool nee, float3& L) {
    float w = 1.0f;
    if (nee && bt.w > 0.0f) {
        const V3 e0 = v3(v0.x, v0.y, v0.z);
        const V3 nl = cross3(sub3(v3(v1.x, v1.y, v1.z), e0), sub3(v3(v2.x, v2.y, v2.z), e0));
        const V3 d = v3(d4.x, d4.y, d4.z);
        const float dd = dot3(d, d);
        const float cl = fd(fabsf(dot3(nl, d)), fq(fm(dot3(nl, nl), dd)));
        if (cl > 0.0f) {
            const float th = __int_as_float(h.y);
            const float pl = fd(fm(fm(th, th), dd), fm(cl, sc.light_total));
            w = fd(fm(bt.w, bt.w), fa(fm(bt.w, bt.w), fm(pl, pl)));
        }
    }
    L.x = fa(L.x, fm(fm(bt.x, m1.y), w));
    L.y = fa(L.y, fm(fm(bt.y, m1.z), w));
    L.z = fa(L.z, fm(fm(bt.z, m1.w), w));
}

// Replay capture: the ray trace b received (origin with its skip id, direction with tmax),
// the distance it returned and the throughput it carried, at entry di = b * npx + pixel.
__device__ __forceinline__ void capture_trace(const cr_debug& dbg, uint32_t di, const float4 o4, const float4 d4,
                                              const int2 h, const float4 bt) {
    reinterpret_cast<float4*>(dbg.ray)[2 * di + 0] = o4;
    reinterpret_cast<float4*>(dbg.ray)[2 * di + 1] = d4;
    dbg.t[di] = h.x >= 0 ? __int_as_float(h.y) : INFINITY;
    reinterpret_cast<float4*>(dbg.beta)[di] = bt;
}

__device__ __forceinline__ void setup_member(const ShadeArgs& a, const PassArgs& p, const SceneDev& sc, int slot,
                                             Member& mb, float3& L, const float4 bt, const int2 h, const float4 d4,
                                             const float tau) {
    if (a.dbg.prim) a.dbg.prim[(p.bounce - 1) * a.npx + mb.pix] = h.x >= 0 ? __float_as_int(__ldg(&sc.tris[3 * h.x]).w) : -1;
    if (a.dbg.ray) capture_trace(a.dbg, (p.bounce - 1) * a.npx + (uint32_t)mb.pix, a.ray_o[slot], d4, h, bt);
    if (h.x < 0) { // miss: environment
        add_environment(sc, bt, L);
        mb.alive = false;
        return;
    }
    CR_DBG(if (!dbg_in_range(&sc, (uint32_t)h.x, kDbgHit, sc.n_tris)) {
        mb.alive = false;
        return;
    })
    const float4 v0 = __ldg(&sc.tris[3 * h.x + 0]);
    const float4 v1 = __ldg(&sc.tris[3 * h.x + 1]);
    const float4 v2 = __ldg(&sc.tris[3 * h.x + 2]);
    const int mat = __float_as_int(v1.w);
    CR_DBG(if (!dbg_in_range(&sc, (uint32_t)mat, kDbgMat, sc.n_mats)) {
        mb.alive = false;
        return;
    })
    const float4 m0 = __ldg(&sc.mats[2 * mat + 0]);
    const float4 m1 = __ldg(&sc.mats[2 * mat + 1]);
    const uint32_t type = (uint32_t)__float_as_int(m0.x);
    mb.orig = __float_as_int(v0.w);
    if (type == kMatEmitter) {
        add_emission(sc, v0, v1, v2, m1, bt, h, d4, mb.nee, L);
        mb.alive = false;
        return;
    }
    if (mb.final_pass) {
        mb.alive = false;
        return;
    }
    const V3 a0 = v3(v0.x, v0.y, v0.z), a1 = v3(v1.x, v1.y, v1.z), a2 = v3(v2.x, v2.y, v2.z);
    const V3 ng = normalize3(cross3(sub3(a1, a0), sub3(a2, a0)));
    const V3 d = v3(d4.x, d4.y, d4.z);
    mb.front = dot3(ng, d) < 0.0f;
    mb.n = mb.front ? ng : v3(-ng.x, -ng.y, -ng.z);
    frame_from(mb.n, mb.t, mb.b);
    const V3 md = v3(-d.x, -d.y, -d.z);
    mb.wo = v3(dot3(md, mb.t), dot3(md, mb.b), dot3(md, mb.n));
    // transmission (the paper's future work, Sec. 6): a Lambertian transmitter joins the
    // diffuse class with its lobe in the lower hemisphere; a smooth dielectric is specular
    mb.cls = (type == kMatLambert || type == kMatTranslucent) ? kClsDiffuse : kClsGlossy;
    // roughness threshold of the classes (a reading: Sec. 3.2 classifies by material): a
    // rough GGX point joins the diffuse class, and while reusing it samples a cosine lobe
    const bool rough_cls = type == kMatGGX && tau > 0.0f && m1.x >= tau;
    if (rough_cls) mb.cls = kClsDiffuse;
    mb.cosgl = rough_cls && (mb.reuse || mb.world);
    mb.hemi = type == kMatTranslucent ? -1.0f : 1.0f;
    mb.type = type;
    mb.rough = m1.x;
    mb.albedo[0] = m0.y;
    mb.albedo[1] = m0.z;
    mb.albedo[2] = m0.w;
    // the member's own BSDF sample, drawn from its pixel's stream
    const uint4 r = philox_seed(mb.seed, (uint32_t)mb.pix, mb.frame, mb.bounce, kTagBsdf);
    const float u1 = unit24(r.x), u2 = unit24(r.y);
    if (type == kMatLambert) {
        mb.wl = sample_cosine(u1, u2);
        mb.w[0] = m0.y;
        mb.w[1] = m0.z;
        mb.w[2] = m0.w;
        mb.valid = true;
    } else if (mb.cosgl) { // a GGX point of the diffuse class: cosine sample, weight pi f
        mb.wl = sample_cosine(u1, u2);
        rough_weight(mb, mb.wl);
    } else if (type == kMatGGX) {
        mb.valid = sample_ggx(mb.wo, m1.x, mb.albedo, u1, u2, mb.wl, mb.w);
    } else if (type == kMatTranslucent) {
        const V3 c = sample_cosine(u1, u2);
        mb.wl = v3(c.x, c.y, -c.z);
        mb.w[0] = m0.y;
        mb.w[1] = m0.z;
        mb.w[2] = m0.w;
        mb.valid = true;
    } else if (type == kMatDielectric) {
        mb.wl = sample_dielectric(mb.wo, m1.x, mb.front, u1);
        mb.w[0] = m0.y;
        mb.w[1] = m0.z;
        mb.w[2] = m0.w;
        mb.valid = mb.wo.z > 0.0f;
    } else {
        mb.wl = v3(-mb.wo.x, -mb.wo.y, mb.wo.z);
        mb.w[0] = m0.y;
        mb.w[1] = m0.z;
        mb.w[2] = m0.w;
        mb.valid = mb.wo.z > 0.0f;
    }
}

// A shared tangent-space direction taken into the member's own diffuse lobe: the normal
// component becomes hemi * |z| (a translucent member mirrors it through the tangent plane),
// so a cosine-distributed direction stays cosine-distributed in either lobe.
__device__ __forceinline__ void take_dir(Member& mb, V3 wl) {
    mb.wl = v3(wl.x, wl.y, fm(mb.hemi, fabsf(wl.z)));
    if (mb.cosgl) {
        rough_weight(mb, mb.wl);
        return;
    }
    mb.w[0] = mb.albedo[0]; // Lambert: f cos / p_cos = albedo
    mb.w[1] = mb.albedo[1];
    mb.w[2] = mb.albedo[2];
    mb.valid = true;
}

// Sec. 3.1 ablation: a world-space direction re-expressed in the member's frame is taken as
// is; outside the member's lobe f = 0 and the path ends.
__device__ __forceinline__ void take_dir_world(Member& mb, V3 l) {
    mb.wl = l;
    if (mb.cosgl) {
        rough_weight(mb, l);
        return;
    }
    mb.w[0] = mb.albedo[0];
    mb.w[1] = mb.albedo[1];
    mb.w[2] = mb.albedo[2];
    mb.valid = fm(mb.hemi, l.z) > 0.0f;
}

// Spawn point of the slot's next ray: p = o + t d, offset by 2^-18 max(1, |p|_inf) along the
// shading normal n (pass -n for a transmitted ray) so that the new ray clears the surface.
__device__ __forceinline__ V3 spawn_point(const ShadeArgs& a, int slot, V3 n) {
    const float4 o4 = a.ray_o[slot];
    const float4 d4 = a.ray_d[slot];
    const float th = __int_as_float(a.hit[slot].y);
    const float px = o4.x + th * d4.x, py = o4.y + th * d4.y, pz = o4.z + th * d4.z;
    const float amax = fmaxf(1.0f, fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz))));
    const float eps = 0x1.0p-18f * amax;
    return v3(px + eps * n.x, py + eps * n.y, pz + eps * n.z);
}

// Solid-angle density with which the member's own BSDF draws the tangent-space direction
// wl: cos / pi (Lambert), the GGX reflection density, 0 for the mirror's delta.
__device__ __forceinline__ float own_pdf(const Member& mb, V3 wl) {
    if (mb.type == kMatLambert) return wl.z > 0.0f ? fm(wl.z, 0.318309886f) : 0.0f;
    if (mb.type == kMatTranslucent) return wl.z < 0.0f ? fm(-wl.z, 0.318309886f) : 0.0f;
    if (mb.cosgl) return wl.z > 0.0f ? fm(wl.z, 0.318309886f) : 0.0f;
    if (mb.type == kMatGGX) return pdf_ggx(mb.wo, wl, mb.rough);
    return 0.0f;
}

// Next-event estimation at a shading point that is not a mirror (a standard estimator the
// paper does not discuss): one emitter point chosen by area, p_A = 1 / A, and the shadow ray
// from the spawn point toward it (direction p - o, ending at 1 - 2^-10 of the way).  The
// contribution w_l beta f Le cos_i cos_l A / r^2 is added by the shadow kernel if the ray is
// unblocked; w_l = p_l^2 / (p_l^2 + p_b^2) is the power-heuristic weight of the light sample
// (p_l = r^2 / (cos_l A), p_b = own_pdf).  Every active position writes its slot's record
// (w < 0: no shadow ray).
__device__ __forceinline__ void next_event(const ShadeArgs& a, const PassArgs& p, int slot, const Member& mb,
                                           const float4 bt, int light_pix) {
    float4 dr = make_float4(0.0f, 0.0f, 0.0f, -1.0f);
    if (mb.alive && mb.nee && mb.type != kMatMirror && mb.type != kMatDielectric) {
        const SceneDev& sc = a.scenes[mb.scene];
        if (sc.n_lights > 0) {
            const uint4 r = philox_seed(mb.seed, (uint32_t)light_pix, mb.frame, mb.bounce, kTagLight);
            const float u0 = unit24(r.x), u1 = unit24(r.y), u2 = unit24(r.z);
            // the first emitter whose running area exceeds u0 * A (the last if none)
            const float x = fm(u0, sc.light_total);
            uint32_t lo = 0, hi = sc.n_lights;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (x < __ldg(&sc.light_cdf[mid])) hi = mid;
                else lo = mid + 1;
            }
            const uint32_t li = lo < sc.n_lights ? lo : sc.n_lights - 1;
            const float4 l0 = __ldg(&sc.lights[4 * li + 0]);
            const float4 l1 = __ldg(&sc.lights[4 * li + 1]);
            const float4 l2 = __ldg(&sc.lights[4 * li + 2]);
            const float4 le = __ldg(&sc.lights[4 * li + 3]);
            const float sq = fq(u1);
            const float b0 = fs(1.0f, sq), b1 = fm(sq, fs(1.0f, u2)), b2 = fm(sq, u2);
            const V3 pl = v3(fa(fa(fm(l0.x, b0), fm(l1.x, b1)), fm(l2.x, b2)),
                             fa(fa(fm(l0.y, b0), fm(l1.y, b1)), fm(l2.y, b2)),
                             fa(fa(fm(l0.z, b0), fm(l1.z, b1)), fm(l2.z, b2)));
            // leave on the side of the lobe (below the surface for a translucent point)
            const V3 o = spawn_point(a, slot, v3(fm(mb.hemi, mb.n.x), fm(mb.hemi, mb.n.y), fm(mb.hemi, mb.n.z)));
            const V3 dl = sub3(pl, o);
            const float r2 = dot3(dl, dl);
            const float rl = fq(r2);
            const float ci = fm(mb.hemi, fd(dot3(mb.n, dl), rl));
            const V3 a0 = v3(l0.x, l0.y, l0.z);
            const V3 nl = cross3(sub3(v3(l1.x, l1.y, l1.z), a0), sub3(v3(l2.x, l2.y, l2.z), a0));
            const float cl = fd(fabsf(dot3(nl, dl)), fm(fq(dot3(nl, nl)), rl));
            if (r2 > 0.0f && ci > 0.0f && cl > 0.0f) {
                const V3 wi = v3(fd(dl.x, rl), fd(dl.y, rl), fd(dl.z, rl));
                const V3 wil = v3(dot3(wi, mb.t), dot3(wi, mb.b), dot3(wi, mb.n));
                float f[3];
                if (mb.type == kMatLambert || mb.type == kMatTranslucent) {
                    f[0] = fm(mb.albedo[0], 0.318309886f);
                    f[1] = fm(mb.albedo[1], 0.318309886f);
                    f[2] = fm(mb.albedo[2], 0.318309886f);
                } else {
                    eval_ggx(mb.wo, wil, mb.rough, mb.albedo, f);
                }
                const float pl = fd(r2, fm(cl, sc.light_total));
                const float pb = own_pdf(mb, wil);
                const float wlt = fd(fm(pl, pl), fa(fm(pl, pl), fm(pb, pb)));
                const float g = fm(fm(fd(fm(ci, cl), r2), sc.light_total), wlt);
                a.shadow_o[slot] = make_float4(o.x, o.y, o.z, __int_as_float(mb.orig));
                a.shadow_c[slot] = make_float4(fm(fm(fm(bt.x, f[0]), le.x), g), fm(fm(fm(bt.y, f[1]), le.y), g),
                                               fm(fm(fm(bt.z, f[2]), le.z), g), 0.0f);
                dr = make_float4(dl.x, dl.y, dl.z, 1.0f - 0x1.0p-10f);
            }
        }
    }
    a.shadow_d[slot] = dr;
}

// Returns whether the path continues (its slot is alive for the next trace).
__device__ __forceinline__ bool finish_member(const ShadeArgs& a, const PassArgs& p, int slot, Member& mb,
                                              float3 L, float4 bt, bool was_alive, int cat) {
    if (a.dbg.cat && mb.pix >= 0 && !mb.final_pass) {
        const uint32_t di = (p.bounce - 1) * a.npx + (uint32_t)mb.pix;
        a.dbg.cat[di] = (uint8_t)cat;
        a.dbg.cls[di] = (uint8_t)(!mb.alive ? kClsNone : (mb.hemi < 0.0f ? 3 : mb.cls)); // 3: translucent
        a.dbg.flags[di] = (uint8_t)((mb.alive ? 1 : 0) | (mb.alive && mb.valid ? 2 : 0));
        V3 lw = v3(0.0f, 0.0f, 0.0f), ww = v3(0.0f, 0.0f, 0.0f);
        if (mb.alive) {
            lw = mb.wl;
            ww = local_to_world(mb.t, mb.b, mb.n, mb.wl);
        }
        a.dbg.local[3 * di + 0] = lw.x;
        a.dbg.local[3 * di + 1] = lw.y;
        a.dbg.local[3 * di + 2] = lw.z;
        a.dbg.world[3 * di + 0] = ww.x;
        a.dbg.world[3 * di + 1] = ww.y;
        a.dbg.world[3 * di + 2] = ww.z;
    }
    if (!was_alive) return false;
    a.radiance[slot] = make_float4(L.x, L.y, L.z, 0.0f);
    if (mb.alive && mb.valid) {
        const V3 o = spawn_point(a, slot, mb.wl.z < 0.0f ? v3(-mb.n.x, -mb.n.y, -mb.n.z) : mb.n);
        const V3 dw = local_to_world(mb.t, mb.b, mb.n, mb.wl);
        a.ray_o[slot] = make_float4(o.x, o.y, o.z, __int_as_float(mb.orig));
        a.ray_d[slot] = make_float4(dw.x, dw.y, dw.z, INFINITY);
        // beta.w: density of the new direction for the MIS weight of the emission it may
        // meet (next-event estimation only; 0 = mirror)
        a.beta[slot] = make_float4(fm(bt.x, mb.w[0]), fm(bt.y, mb.w[1]), fm(bt.z, mb.w[2]),
                                   mb.nee ? own_pdf(mb, mb.wl) : 0.0f);
        a.alive[slot] = 1;
        return true;
    }
    a.alive[slot] = 0;
    return false;
}

// Queue compaction inside the shade (the default): after shading, each block appends its
// continuing slots to the ray queue and its groups with a continuing member to the group
// queue, in position order, at ranges it reserves with one atomic add per queue.  Groups
// keep their K slots together and a block's slots stay adjacent; the blocks' ranges follow
// their completion order, so the queue order (not the result of any slot) can differ from
// run to run.  CR_OPT_ORDERED_QUEUES uses the three-launch order-preserving compaction.
template <uint32_t kThreads>
__device__ __forceinline__ void append_queues(const ShadeArgs& a, uint32_t K, int slot, bool alive, bool group_head) {
    __shared__ unsigned long long s_w[kThreads / 32];
    __shared__ unsigned long long s_base;
    constexpr uint32_t nw = kThreads / 32;
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    // block-exclusive ranks of (ray, group), packed as rays | groups << 32
    const unsigned long long v = (alive ? 1ull : 0ull) | (group_head ? 1ull << 32 : 0ull);
    unsigned long long x = v;
    for (uint32_t off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = lane < nw ? s_w[lane] : 0ull;
        for (uint32_t off = 1; off < nw; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += y;
        }
        if (lane < nw) s_w[lane] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long agg = s_w[nw - 1];
        const uint32_t nr = (uint32_t)agg, ng = (uint32_t)(agg >> 32);
        uint32_t br = 0, bg = 0;
        if (nr) {
            br = atomicAdd(&a.queue_counts[0], nr);
            atomicAdd(a.rays_queued, (unsigned long long)nr);
        }
        if (ng) bg = atomicAdd(&a.queue_counts[1], ng);
        s_base = (unsigned long long)br | ((unsigned long long)bg << 32);
    }
    __syncthreads();
    const unsigned long long rank = x - v + (w > 0 ? s_w[w - 1] : 0ull);
    const uint32_t qr = (uint32_t)s_base + (uint32_t)rank, qg = (uint32_t)(s_base >> 32) + (uint32_t)(rank >> 32);
    if (alive) {
        if (qr < a.ray_cap) a.ray_queue[qr] = slot;
        else atomicOr(a.queue_err, 1u);
    }
    if (group_head) {
        if (qg < a.group_cap) a.group_queue_out[qg] = slot / (int)K;
        else atomicOr(a.queue_err, 1u);
    }
}

// K <= 32: a group is a K-lane segment of a warp; votes by ballot, the donor's direction by
// shuffle, the hybrid sum by an xor butterfly (which equals the pairwise tree sum in every
// lane because float addition is commutative).
#ifndef CR_SHADE_MIN_BLOCKS
#define CR_SHADE_MIN_BLOCKS 8 // registers sized for 8 resident 128-thread blocks per SM (0: no cap)
#endif
#ifndef CR_SHADE_WARP_BLOCK
// threads per block of the K <= 32 shade kernel: 256 and 512 give longer appended queue
// ranges (secondary trace 0.6-1% faster) but a slower shade; the step is within 0.4% either way
#define CR_SHADE_WARP_BLOCK 128
#endif
#if CR_SHADE_MIN_BLOCKS
__global__ void __launch_bounds__(CR_SHADE_WARP_BLOCK, CR_SHADE_MIN_BLOCKS * 128 / CR_SHADE_WARP_BLOCK)
    k_shade_warp(ShadeArgs a, PassArgs p) {
#else
__global__ void k_shade_warp(ShadeArgs a, PassArgs p) {
#endif
    const uint32_t K = p.k;
    const uint32_t n_groups = a.group_queue ? min(*a.group_count, a.n_groups_max) : a.n_groups_max;
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t gq = pos / K, lane_g = pos % K;
    const bool active = gq < n_groups;
    int slot = -1;
    Member mb;
    mb.pix = -1;
    mb.alive = false;
    mb.cls = kClsNone;
    mb.valid = false;
    mb.wl = v3(0.0f, 0.0f, 0.0f);
    bool was_alive = false;
    float4 bt = make_float4(0, 0, 0, 0);
    float3 L = make_float3(0, 0, 0);
    mb.final_pass = true;
    mb.bounce = p.bounce;
    mb.reuse = false;
    mb.world = false;
    mb.nee = false;
    mb.nee_shared = false;
    mb.hdonor = false;
    mb.cosgl = false;
    mb.type = kMatLambert;
    mb.hemi = 1.0f;
    mb.front = true;
    if (active) {
        const uint32_t g = a.group_queue ? (uint32_t)a.group_queue[gq] : gq;
        slot = (int)(g * K + lane_g);
        // the slot's state in one round of independent loads (read even for slots that turn
        // out dead, which takes them off the dependency chain of the live ones)
        mb.pix = a.pixel[slot];
        const uint32_t jid = a.slot_job[slot];
        const bool alive_in = a.alive[slot] != 0;
        const int2 h = a.hit[slot];
        const float4 d4 = a.ray_d[slot];
        const float4 b4 = a.beta[slot];
        const float4 r4 = a.radiance[slot];
        const JobDev* Jp = nullptr;
        if (mb.pix >= 0) { // every valid slot knows whether its job is past its last bounce
            Jp = &a.jobs[jid];
            mb.bounce = p.rolling ? Jp->step : p.bounce;
            mb.final_pass = mb.bounce > Jp->max_bounces;
            mb.reuse = (Jp->reuse_mask >> mb.bounce) & 1u;
            mb.world = (Jp->world_mask >> mb.bounce) & 1u;
            mb.nee = Jp->nee != 0;
            mb.nee_shared = Jp->nee == 2u;
            mb.hdonor = Jp->hybrid_donor != 0;
            mb.scene = Jp->scene;
            mb.seed = Jp->seed;
            mb.frame = Jp->frame;
        }
        was_alive = mb.pix >= 0 && alive_in;
        if (was_alive) {
            const JobDev& J = *Jp;
            mb.alive = true;
            bt = b4;
            L = make_float3(r4.x, r4.y, r4.z);
            setup_member(a, p, a.scenes[J.scene], slot, mb, L, bt, h, d4, J.diffuse_rough);
        }
    }
    int cat = kCatEmpty;
    int light_pix = mb.pix;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t seg = lane & ~(K - 1u);
    const uint32_t segmask = K == 32u ? 0xffffffffu : (((1u << K) - 1u) << seg);
    {
        // shared light samples: the group's first alive member owns the light stream
        if (__any_sync(0xffffffffu, mb.nee_shared)) {
            const uint32_t bal = __ballot_sync(0xffffffffu, mb.alive) & segmask;
            const int owner = bal ? __ffs(bal) - 1 : (int)lane;
            const int opix = __shfl_sync(0xffffffffu, mb.pix, owner);
            if (mb.nee_shared) light_pix = opix;
        }
        const uint32_t bd = __ballot_sync(0xffffffffu, mb.alive && mb.cls == kClsDiffuse) & segmask;
        const uint32_t bg = __ballot_sync(0xffffffffu, mb.alive && mb.cls == kClsGlossy) & segmask;
        cat = bd && bg ? kCatHybrid : (bd ? kCatDiffuse : (bg ? kCatGlossy : kCatEmpty));
        // reuse is uniform within a group (one job); the shuffles run in every lane of a
        // warp that has any reusing lane
        if (__any_sync(0xffffffffu, mb.reuse)) {
            const int donor = bd ? __ffs(bd) - 1 : (int)lane;
            const V3 wd = v3(__shfl_sync(0xffffffffu, mb.wl.x, donor), __shfl_sync(0xffffffffu, mb.wl.y, donor),
                             __shfl_sync(0xffffffffu, mb.wl.z, donor));
            const bool contrib = mb.alive && mb.cls == kClsGlossy && mb.valid;
            V3 s = contrib ? mb.wl : v3(0.0f, 0.0f, 0.0f);
            for (uint32_t off = 1; off < K; off <<= 1) {
                const float sx = __shfl_xor_sync(0xffffffffu, s.x, off);
                const float sy = __shfl_xor_sync(0xffffffffu, s.y, off);
                const float sz = __shfl_xor_sync(0xffffffffu, s.z, off);
                s = v3(fa(s.x, sx), fa(s.y, sy), fa(s.z, sz));
            }
            if (mb.reuse && mb.alive && mb.cls == kClsDiffuse) {
                if (cat == kCatDiffuse) {
                    take_dir(mb, wd);
                } else if (cat == kCatHybrid) {
                    const float l2 = dot3(s, s);
                    if (mb.hdonor) {
                        take_dir(mb, wd); // donor option: the first diffuse member's own sample
                    } else if (l2 > 0.0f) {
                        // a rough GGX member keeps its own cosine sample: its weight pi f at
                        // the glossy average (near its specular peak) would be far above 1
                        const float l = fq(l2);
                        if (!mb.cosgl) take_dir(mb, v3(fd(s.x, l), fd(s.y, l), fd(s.z, l)));
                    } else {
                        take_dir(mb, wd); // no valid glossy sample: first diffuse member's
                    }
                }
            }
        }
        // Sec. 3.1 direct reuse (ablation): the first alive member's world-space direction,
        // re-expressed in each diffuse member's frame; below the surface the path ends
        if (__any_sync(0xffffffffu, mb.world)) {
            const uint32_t ba = __ballot_sync(0xffffffffu, mb.alive) & segmask;
            const int wdonor = ba ? __ffs(ba) - 1 : (int)lane;
            const V3 ww = mb.alive ? local_to_world(mb.t, mb.b, mb.n, mb.wl) : v3(0.0f, 0.0f, 0.0f);
            const V3 wdw = v3(__shfl_sync(0xffffffffu, ww.x, wdonor), __shfl_sync(0xffffffffu, ww.y, wdonor),
                              __shfl_sync(0xffffffffu, ww.z, wdonor));
            const bool dvalid = __shfl_sync(0xffffffffu, mb.valid ? 1 : 0, wdonor) != 0;
            if (mb.world && mb.alive && mb.cls == kClsDiffuse && ba && dvalid) {
                take_dir_world(mb, v3(dot3(wdw, mb.t), dot3(wdw, mb.b), dot3(wdw, mb.n)));
            }
        }
    }
    if (active && a.shadow_d) next_event(a, p, slot, mb, bt, light_pix);
    const bool next_alive = active && finish_member(a, p, slot, mb, L, bt, was_alive, cat);
    if (a.ray_queue) {
        // groups are K-lane segments of a warp: a group continues if any member does
        const uint32_t nb = __ballot_sync(0xffffffffu, next_alive) & segmask;
        append_queues<CR_SHADE_WARP_BLOCK>(a, K, slot, next_alive, lane == seg && nb != 0u);
    }
}

#ifndef CR_SHADE_BLOCK_MIN_BLOCKS
// registers sized for 4 resident 256-thread blocks per SM (64 per thread): 12-18% less shade
// time at K = 64 and 256 than the uncapped 79 registers (3 blocks); caps for 3 or 5 blocks
// do worse
#define CR_SHADE_BLOCK_MIN_BLOCKS 4
#endif
// 32 < K <= 256: a group spans K/32 warps of a 256-thread block; per-warp ballots and the
// members' samples go through shared memory and the hybrid sum is a pairwise tree over the
// group's slots.
__global__ void __launch_bounds__(256, CR_SHADE_BLOCK_MIN_BLOCKS) k_shade_block(ShadeArgs a, PassArgs p) {
    __shared__ uint32_t s_bd[8], s_bg[8], s_ba[8];
    __shared__ float s_own[3][256];
    __shared__ float s_sum[3][256];
    __shared__ float s_world[4][256]; // world-space direction and validity (Sec. 3.1 ablation)
    __shared__ int s_pix[256];        // members' pixels (owner of a shared light sample)
    __shared__ uint32_t s_next[8];    // per-warp ballots of the slots that continue
    const uint32_t K = p.k;
    const uint32_t n_groups = a.group_queue ? min(*a.group_count, a.n_groups_max) : a.n_groups_max;
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t gq = pos / K, lane_g = pos % K;
    const bool active = gq < n_groups;
    int slot = -1;
    Member mb;
    mb.pix = -1;
    mb.alive = false;
    mb.cls = kClsNone;
    mb.valid = false;
    mb.wl = v3(0.0f, 0.0f, 0.0f);
    bool was_alive = false;
    float4 bt = make_float4(0, 0, 0, 0);
    float3 L = make_float3(0, 0, 0);
    mb.final_pass = true;
    mb.bounce = p.bounce;
    mb.reuse = false;
    mb.world = false;
    mb.nee = false;
    mb.nee_shared = false;
    mb.hdonor = false;
    mb.cosgl = false;
    mb.type = kMatLambert;
    mb.hemi = 1.0f;
    mb.front = true;
    if (active) {
        const uint32_t g = a.group_queue ? (uint32_t)a.group_queue[gq] : gq;
        slot = (int)(g * K + lane_g);
        // the slot's state in one round of independent loads (read even for slots that turn
        // out dead, which takes them off the dependency chain of the live ones)
        mb.pix = a.pixel[slot];
        const uint32_t jid = a.slot_job[slot];
        const bool alive_in = a.alive[slot] != 0;
        const int2 h = a.hit[slot];
        const float4 d4 = a.ray_d[slot];
        const float4 b4 = a.beta[slot];
        const float4 r4 = a.radiance[slot];
        const JobDev* Jp = nullptr;
        if (mb.pix >= 0) { // every valid slot knows whether its job is past its last bounce
            Jp = &a.jobs[jid];
            mb.bounce = p.rolling ? Jp->step : p.bounce;
            mb.final_pass = mb.bounce > Jp->max_bounces;
            mb.reuse = (Jp->reuse_mask >> mb.bounce) & 1u;
            mb.world = (Jp->world_mask >> mb.bounce) & 1u;
            mb.nee = Jp->nee != 0;
            mb.nee_shared = Jp->nee == 2u;
            mb.hdonor = Jp->hybrid_donor != 0;
            mb.scene = Jp->scene;
            mb.seed = Jp->seed;
            mb.frame = Jp->frame;
        }
        was_alive = mb.pix >= 0 && alive_in;
        if (was_alive) {
            const JobDev& J = *Jp;
            mb.alive = true;
            bt = b4;
            L = make_float3(r4.x, r4.y, r4.z);
            setup_member(a, p, a.scenes[J.scene], slot, mb, L, bt, h, d4, J.diffuse_rough);
        }
    }
    int cat = kCatEmpty;
    int light_pix = mb.pix;
    {
        const uint32_t t = threadIdx.x, w = t >> 5;
        s_pix[t] = mb.pix;
        const uint32_t bd = __ballot_sync(0xffffffffu, mb.alive && mb.cls == kClsDiffuse);
        const uint32_t bg = __ballot_sync(0xffffffffu, mb.alive && mb.cls == kClsGlossy);
        const uint32_t ba = __ballot_sync(0xffffffffu, mb.alive);
        if ((t & 31u) == 0) {
            s_bd[w] = bd;
            s_bg[w] = bg;
            s_ba[w] = ba;
        }
        {
            const V3 ww = mb.alive ? local_to_world(mb.t, mb.b, mb.n, mb.wl) : v3(0.0f, 0.0f, 0.0f);
            s_world[0][t] = ww.x;
            s_world[1][t] = ww.y;
            s_world[2][t] = ww.z;
            s_world[3][t] = mb.valid ? 1.0f : 0.0f;
        }
        const bool contrib = mb.alive && mb.cls == kClsGlossy && mb.valid;
        s_own[0][t] = mb.wl.x;
        s_own[1][t] = mb.wl.y;
        s_own[2][t] = mb.wl.z;
        s_sum[0][t] = contrib ? mb.wl.x : 0.0f;
        s_sum[1][t] = contrib ? mb.wl.y : 0.0f;
        s_sum[2][t] = contrib ? mb.wl.z : 0.0f;
        __syncthreads();
        const uint32_t gbase = (t / K) * K; // first thread of the group in the block
        bool any_d = false, any_g = false;
        int donor = -1;
        for (uint32_t ww = gbase >> 5; ww < (gbase + K) >> 5; ++ww) {
            if (s_bd[ww] && donor < 0) donor = (int)(ww * 32u + __ffs(s_bd[ww]) - 1);
            any_d |= s_bd[ww] != 0;
            any_g |= s_bg[ww] != 0;
        }
        cat = any_d && any_g ? kCatHybrid : (any_d ? kCatDiffuse : (any_g ? kCatGlossy : kCatEmpty));
        if (__syncthreads_or(mb.reuse)) {
            for (uint32_t stride = 1; stride < K; stride <<= 1) {
                if ((t - gbase) % (2u * stride) == 0) {
                    s_sum[0][t] = fa(s_sum[0][t], s_sum[0][t + stride]);
                    s_sum[1][t] = fa(s_sum[1][t], s_sum[1][t + stride]);
                    s_sum[2][t] = fa(s_sum[2][t], s_sum[2][t + stride]);
                }
                __syncthreads();
            }
            if (mb.reuse && mb.alive && mb.cls == kClsDiffuse) {
                const V3 wd = v3(s_own[0][donor], s_own[1][donor], s_own[2][donor]);
                if (cat == kCatDiffuse) {
                    take_dir(mb, wd);
                } else if (cat == kCatHybrid) {
                    const V3 s = v3(s_sum[0][gbase], s_sum[1][gbase], s_sum[2][gbase]);
                    const float l2 = dot3(s, s);
                    if (mb.hdonor) {
                        take_dir(mb, wd); // donor option: the first diffuse member's own sample
                    } else if (l2 > 0.0f) {
                        const float l = fq(l2); // rough GGX members keep their own cosine sample
                        if (!mb.cosgl) take_dir(mb, v3(fd(s.x, l), fd(s.y, l), fd(s.z, l)));
                    } else {
                        take_dir(mb, wd);
                    }
                }
            }
        }
        if (mb.world && mb.alive && mb.cls == kClsDiffuse) {
            int wdonor = -1;
            for (uint32_t ww = gbase >> 5; ww < (gbase + K) >> 5 && wdonor < 0; ++ww)
                if (s_ba[ww]) wdonor = (int)(ww * 32u + __ffs(s_ba[ww]) - 1);
            if (wdonor >= 0 && s_world[3][wdonor] != 0.0f) {
                const V3 wdw = v3(s_world[0][wdonor], s_world[1][wdonor], s_world[2][wdonor]);
                take_dir_world(mb, v3(dot3(wdw, mb.t), dot3(wdw, mb.b), dot3(wdw, mb.n)));
            }
        }
        if (mb.nee_shared) { // the group's first alive member owns the light stream
            int owner = -1;
            for (uint32_t ww = gbase >> 5; ww < (gbase + K) >> 5 && owner < 0; ++ww)
                if (s_ba[ww]) owner = (int)(ww * 32u + __ffs(s_ba[ww]) - 1);
            if (owner >= 0) light_pix = s_pix[owner];
        }
    }
    if (active && a.shadow_d) next_event(a, p, slot, mb, bt, light_pix);
    const bool next_alive = active && finish_member(a, p, slot, mb, L, bt, was_alive, cat);
    if (a.ray_queue) {
        // a group spans K/32 warps of the block: OR of their ballots
        const uint32_t t = threadIdx.x;
        const uint32_t nb = __ballot_sync(0xffffffffu, next_alive);
        if ((t & 31u) == 0) s_next[t >> 5] = nb;
        __syncthreads();
        bool head = false;
        if (t % K == 0)
            for (uint32_t ww = t >> 5; ww < (t + K) >> 5; ++ww) head |= s_next[ww] != 0u;
        append_queues<256>(a, K, slot, next_alive, head);
    }
}

// ------------------------------------------------------------------------------------
// Order-preserving group-granular compaction (CR_OPT_ORDERED_QUEUES; the default appends in
// the shade instead).  Positions [0, n_groups*K) of the last shade (group queue order) are
// scanned in blocks of 256; a group survives if any member is alive and keeps its K slots
// together in the group queue, while the ray queue lists the alive slots.  Three launches
// (count, scan, scatter) keep the whole queue in position order.
constexpr uint32_t kCompactBlock = 256;

__device__ __forceinline__ void position_info(const int32_t* gq_in, uint32_t n_groups, uint32_t K, uint32_t pos,
                                              const uint8_t* alive, int& slot, bool& a) {
    slot = -1;
    a = false;
    const uint32_t g = pos / K;
    if (g < n_groups) {
        const uint32_t grp = gq_in ? (uint32_t)gq_in[g] : g;
        slot = (int)(grp * K + pos % K);
        a = alive[slot] != 0;
    }
}


__global__ void __launch_bounds__(kCompactBlock) k_compact_count(const int32_t* gq_in, const uint32_t* n_groups_ptr,
                                                                 uint32_t n_groups_max, uint32_t K,
                                                                 const uint8_t* __restrict__ alive,
                                                                 uint32_t* __restrict__ block_counts) {
    __shared__ uint8_t s_alive[kCompactBlock];
    const uint32_t n_groups = n_groups_ptr ? min(*n_groups_ptr, n_groups_max) : n_groups_max;
    const uint32_t pos = blockIdx.x * kCompactBlock + threadIdx.x;
    int slot;
    bool a;
    position_info(gq_in, n_groups, K, pos, alive, slot, a);
    s_alive[threadIdx.x] = a;
    __syncthreads();
    uint32_t gl = 0;
    if (threadIdx.x % K == 0) {
        for (uint32_t j = 0; j < K; ++j) gl |= s_alive[threadIdx.x + j];
    }
    const uint32_t tot_r = (uint32_t)__syncthreads_count(a);
    const uint32_t tot_g = (uint32_t)__syncthreads_count(gl != 0u);
    if (threadIdx.x == 0) {
        block_counts[2 * blockIdx.x + 0] = tot_r;
        block_counts[2 * blockIdx.x + 1] = tot_g;
    }
}

// Exclusive scan of the per-block counts in one block; totals go to out_counts[0..1] and are
// added to the running statistics.
__global__ void __launch_bounds__(1024) k_compact_scan(uint32_t* __restrict__ block_counts, uint32_t n_blocks,
                                                       uint32_t* __restrict__ out_counts,
                                                       unsigned long long* __restrict__ stat) {
    // both columns at once: each thread loads its run of (rays, groups) pairs as 8-byte
    // words (independent loads), the two counts travel packed in one 64-bit value through
    // the block scan (each column total < 2^32)
    __shared__ unsigned long long s_w[32];
    uint2* bc = reinterpret_cast<uint2*>(block_counts);
    const uint32_t per = (n_blocks + blockDim.x - 1) / blockDim.x;
    const uint32_t b0 = threadIdx.x * per;
    unsigned long long local = 0;
    for (uint32_t k = 0; k < per; ++k)
        if (b0 + k < n_blocks) {
            const uint2 v = bc[b0 + k];
            local += (unsigned long long)v.x | ((unsigned long long)v.y << 32);
        }
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    unsigned long long x = local;
    for (uint32_t off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const uint32_t nw = blockDim.x >> 5;
        unsigned long long t = lane < nw ? s_w[lane] : 0ull;
        for (uint32_t off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += y;
        }
        if (lane < nw) s_w[lane] = t;
    }
    __syncthreads();
    unsigned long long run = x - local + (w > 0 ? s_w[w - 1] : 0ull);
    for (uint32_t k = 0; k < per; ++k)
        if (b0 + k < n_blocks) {
            const uint2 v = bc[b0 + k];
            bc[b0 + k] = make_uint2((uint32_t)run, (uint32_t)(run >> 32));
            run += (unsigned long long)v.x | ((unsigned long long)v.y << 32);
        }
    if (threadIdx.x == 0) {
        const unsigned long long total = s_w[(blockDim.x >> 5) - 1];
        out_counts[0] = (uint32_t)total;
        out_counts[1] = (uint32_t)(total >> 32);
        if (stat) atomicAdd(stat, (unsigned long long)(uint32_t)total);
    }
}

__global__ void __launch_bounds__(kCompactBlock) k_compact_scatter(const int32_t* gq_in, const uint32_t* n_groups_ptr,
                                                                   uint32_t n_groups_max, uint32_t K,
                                                                   const uint8_t* __restrict__ alive,
                                                                   const uint32_t* __restrict__ block_offsets,
                                                                   int32_t* __restrict__ ray_queue,
                                                                   int32_t* __restrict__ gq_out) {
    __shared__ uint8_t s_alive[kCompactBlock];
    __shared__ uint32_t s_warp[32];
    const uint32_t n_groups = n_groups_ptr ? min(*n_groups_ptr, n_groups_max) : n_groups_max;
    const uint32_t pos = blockIdx.x * kCompactBlock + threadIdx.x;
    int slot;
    bool a;
    position_info(gq_in, n_groups, K, pos, alive, slot, a);
    s_alive[threadIdx.x] = a;
    __syncthreads();
    uint32_t gl = 0;
    if (threadIdx.x % K == 0) {
        for (uint32_t j = 0; j < K; ++j) gl |= s_alive[threadIdx.x + j];
    }
    uint32_t tot;
    const uint32_t rr = block_excl_scan(a ? 1u : 0u, s_warp, tot);
    const uint32_t rg = block_excl_scan(gl, s_warp, tot);
    if (a) ray_queue[block_offsets[2 * blockIdx.x] + rr] = slot;
    if (gl) gq_out[block_offsets[2 * blockIdx.x + 1] + rg] = slot / (int)K;
}

// ------------------------------------------------------------------------------------
// Reordering comparators (Table 1): a 30-bit key per ray, then a stable LSD radix sort of
// (key, slot).  Positions are quantised in the scene box; directions through the octahedral
// map of the unit sphere onto [-1,1]^2.  Keys (the paper cites their sources without giving
// bit layouts; these layouts are our readings):
//   0 TwoPoint     5 bits of each coordinate of the origin and of the point 0.25 x (largest
//                  scene extent) along the ray, interleaved (6-D Morton)
//   1 Origin       10 bits per origin coordinate (3-D Morton)
//   2 Reis         origin (6 bits per coordinate, 3-D Morton) above direction (6 bits per
//                  octahedral coordinate, 2-D Morton)
//   3 Costa        the same fields with the direction above the origin
//   4 AilaCompact  origin and direction interleaved (5-D Morton, 6 bits per coordinate)
//   5 HierarchyCut a key from the acceleration structure, our reading of MLHCC (the paper
//                  describes it only as a code from cuts of the BVH, length 32, with
//                  lambda = 0.125): the cut at depth l is the set of BVH2 nodes of depth l, and
//                  a point's code at that level is the child its descent takes (1 bit).  The
//                  origin and the point lambda x (largest scene extent) along the ray are
//                  located by descending from the root to the nearest child box, and their
//                  15-level paths are interleaved, origin first, top level most significant
//                  (30 bits, the width of the sort's keys)
constexpr uint32_t kHcutLevels = 15;
constexpr float kHcutLambda = 0.125f;

__device__ __forceinline__ float box_dist2(float px, float py, float pz, float lox, float hix, float loy, float hiy,
                                           float loz, float hiz) {
    const float dx = fmaxf(fmaxf(lox - px, px - hix), 0.0f);
    const float dy = fmaxf(fmaxf(loy - py, py - hiy), 0.0f);
    const float dz = fmaxf(fmaxf(loz - pz, pz - hiz), 0.0f);
    return dx * dx + dy * dy + dz * dz;
}

// Path bits of point p through the BVH2 (root = node 0): at each node the child whose box is
// nearer to p (distance 0 inside), ties (p in both) to the child whose box centre is nearer;
// levels below a leaf add zero bits.
__device__ __forceinline__ uint32_t hcut_path(const float4* __restrict__ nodes, float px, float py, float pz) {
    uint32_t code = 0;
    int node = 0;
    for (uint32_t l = 0; l < kHcutLevels; ++l) {
        code <<= 1;
        if (node < 0) continue;
        const float4 n0 = __ldg(&nodes[4 * node + 0]);
        const float4 n1 = __ldg(&nodes[4 * node + 1]);
        const float4 n2 = __ldg(&nodes[4 * node + 2]);
        const float4 n3 = __ldg(&nodes[4 * node + 3]);
        const float d0 = box_dist2(px, py, pz, n0.x, n0.y, n0.z, n0.w, n2.x, n2.y);
        const float d1 = box_dist2(px, py, pz, n1.x, n1.y, n1.z, n1.w, n2.z, n2.w);
        bool right;
        if (d0 != d1) {
            right = d1 < d0;
        } else {
            const float c0 = box_dist2(px, py, pz, 0.5f * (n0.x + n0.y), 0.5f * (n0.x + n0.y), 0.5f * (n0.z + n0.w),
                                       0.5f * (n0.z + n0.w), 0.5f * (n2.x + n2.y), 0.5f * (n2.x + n2.y));
            const float c1 = box_dist2(px, py, pz, 0.5f * (n1.x + n1.y), 0.5f * (n1.x + n1.y), 0.5f * (n1.z + n1.w),
                                       0.5f * (n1.z + n1.w), 0.5f * (n2.z + n2.w), 0.5f * (n2.z + n2.w));
            right = c1 < c0;
        }
        code |= right ? 1u : 0u;
        node = __float_as_int(right ? n3.y : n3.x);
    }
    return code;
}

__device__ __forceinline__ uint32_t quant(float v, float lo, float scale, uint32_t bits) {
    const float m = (float)((1u << bits) - 1u);
    return (uint32_t)fminf(fmaxf((v - lo) * scale * m, 0.0f), m);
}

// interleave n coordinates of `bits` bits each, coordinate 0 most significant at each level
__device__ __forceinline__ uint32_t interleave(const uint32_t* q, int n, int bits) {
    uint32_t key = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int k = 0; k < n; ++k) key = (key << 1) | ((q[k] >> b) & 1u);
    return key;
}

// The reordering key of one queued ray (30 bits).
__device__ __forceinline__ uint32_t morton_key(const float4* __restrict__ ray_o, const float4* __restrict__ ray_d,
                                               int slot, const SceneDev* __restrict__ scenes,
                                               const uint16_t* __restrict__ slot_scene, uint32_t kind) {
    const SceneDev& sc = scenes[slot_scene[slot]];
    float l[3], s[3], emax = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ext = sc.hi[k] - sc.lo[k];
        l[k] = sc.lo[k];
        s[k] = ext > 0.0f ? 1.0f / ext : 0.0f;
        emax = fmaxf(emax, ext);
    }
    const float4 o = ray_o[slot], d = ray_d[slot];
    const float po[3] = {o.x, o.y, o.z};
    uint32_t key = 0;
    if (kind == 5) {
        const float il = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z) * (kHcutLambda * emax);
        const uint32_t a = hcut_path(sc.nodes2, o.x, o.y, o.z);
        const uint32_t b = hcut_path(sc.nodes2, o.x + d.x * il, o.y + d.y * il, o.z + d.z * il);
        const uint32_t q[2] = {a, b};
        return interleave(q, 2, kHcutLevels);
    }
    if (kind == 0) {
        const float il = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z) * (0.25f * emax);
        const float pe[3] = {o.x + d.x * il, o.y + d.y * il, o.z + d.z * il};
        uint32_t q[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            q[k] = quant(po[k], l[k], s[k], 5);
            q[3 + k] = quant(pe[k], l[k], s[k], 5);
        }
        key = interleave(q, 6, 5);
    } else if (kind == 1) {
        uint32_t q[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) q[k] = quant(po[k], l[k], s[k], 10);
        key = interleave(q, 3, 10);
    } else {
        // octahedral direction coordinates in [-1, 1]
        const float inv = 1.0f / (fabsf(d.x) + fabsf(d.y) + fabsf(d.z));
        float u = d.x * inv, v = d.y * inv;
        if (d.z < 0.0f) {
            const float uu = (1.0f - fabsf(v)) * copysignf(1.0f, u);
            const float vv = (1.0f - fabsf(u)) * copysignf(1.0f, v);
            u = uu;
            v = vv;
        }
        uint32_t qd[2] = {quant(u, -1.0f, 0.5f, 6), quant(v, -1.0f, 0.5f, 6)};
        uint32_t qo[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) qo[k] = quant(po[k], l[k], s[k], 6);
        if (kind == 2) {
            key = (interleave(qo, 3, 6) << 12) | interleave(qd, 2, 6);
        } else if (kind == 3) {
            key = (interleave(qd, 2, 6) << 18) | interleave(qo, 3, 6);
        } else {
            const uint32_t q5[5] = {qo[0], qo[1], qo[2], qd[0], qd[1]};
            key = interleave(q5, 5, 6);
        }
    }
    return key;
}

// ------------------------------------------------------------------------------------
// Stable LSD radix sort of the 30-bit keys with their slots: three passes of 10-bit digits
// after the key kernel, all three in one cooperative launch (k_sort_coop below).  Tiles are
// kOsTile keys; a block ranks a tile's keys stably (warp multisplit by ballots) and scatters
// them through shared memory so that writes of one digit are contiguous.  The grid is one
// wave of resident blocks; the live key count is read on the device.
constexpr uint32_t kRadixBits = 10, kRadix = 1u << kRadixBits, kRadixMask = kRadix - 1u, kRadixPasses = 3;
constexpr uint32_t kOsThreads = 256, kOsWarps = kOsThreads / 32, kOsRounds = 16;
constexpr uint32_t kOsWarpKeys = 32 * kOsRounds, kOsTile = kOsWarps * kOsWarpKeys; // 4096 keys per tile
constexpr uint32_t kCoopMaxGrid = 1024; // blocks of the sort launch at most (chunk sums kept in shared memory)
// sort workspace (uint32 words): word 0 the grid-barrier counter (cleared by the key kernel),
// from kSortF the digit counts F of the live tiles (tiles x kRadix), then kCoopMaxGrid chunk sums
constexpr uint32_t kSortCtr = 0, kSortF = 64;
constexpr uint32_t kSortErrBit = 2u; // error word bit: a grid-barrier wait ran out

__global__ void __launch_bounds__(512) k_morton(const float4* __restrict__ ray_o, const float4* __restrict__ ray_d,
                                                const int32_t* __restrict__ queue, const uint32_t* __restrict__ count,
                                                uint32_t n_max, const SceneDev* __restrict__ scenes,
                                                const uint16_t* __restrict__ slot_scene, uint32_t kind,
                                                uint32_t* __restrict__ keys, int32_t* __restrict__ vals,
                                                int32_t* __restrict__ vals_alt, uint32_t* __restrict__ ctr) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *ctr = 0u; // the sort launch's grid-barrier counter
    const uint32_t n = min(*count, n_max);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int slot;
        uint32_t key;
        if (ray_o) {
            slot = queue[i];
            key = morton_key(ray_o, ray_d, slot, scenes, slot_scene, kind);
        } else { // a caller's keys (queue) and values (slot_scene): the sort alone
            key = reinterpret_cast<const uint32_t*>(queue)[i] & ((1u << (kRadixBits * kRadixPasses)) - 1u);
            slot = reinterpret_cast<const int32_t*>(slot_scene)[i];
        }
        keys[i] = key;
        vals[i] = slot;
        // the other value buffer starts as a copy, so every position a pass can leave
        // unwritten (only after a grid-barrier wait ran out) still holds a valid slot
        vals_alt[i] = slot;
    }
}

// ------------------------------------------------------------------------------------
// The three passes as one cooperative launch.  All blocks are resident at once (a
// cooperative launch guarantees it), so the counts of earlier tiles come from a grid-wide
// scan between two grid barriers; a look-back chain over the tiles' published counts, the
// single-pass alternative, measured slower here (its walk, not the ranking, set a tile's
// latency at ~1M keys).  Per pass:
//   A  each block ranks its tiles' keys stably (warp multisplit, as above), keeps each
//      tile in digit order and writes the tile's digit counts to F[d * T + t]
//      (digit-major, T live tiles);
//   -- grid barrier --
//   B  exclusive scan of F: every block scans one chunk in place and publishes the chunk's
//      sum.  In digit-major order the exclusive prefix of (d, t) is exactly the output
//      position of the first key of digit d in tile t: all keys of smaller digits plus
//      those of digit d in earlier tiles;
//   -- grid barrier --
//   C  each block adds the prefix of the chunk sums and scatters its tiles' keys.
// A block that owns one tile keeps it in shared memory from A to C; with more tiles than
// blocks, A writes each tile back in digit order over its own input range and C reads it
// again.  A further barrier separates the passes.  Every barrier wait is bounded: when one
// runs out the error word is set and the block returns, so the others run out too.
constexpr uint32_t kBarrierSpins = 1u << 21;   // polls of a grid barrier before its wait is given up

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Arrive at the grid barrier whose completion is ctr == target and wait (bounded) for the
// other participating blocks.  Returns false, uniformly over the block, when the wait ran out.  The arrival is a
// release (it publishes every write the block made before its bar.sync, release being
// cumulative) and the poll an acquire, so no full fence is needed on either side.
__device__ __forceinline__ bool grid_barrier(uint32_t* ctr, uint32_t target, uint32_t* err, uint32_t* s_flag) {
    __syncthreads(); // every thread's writes precede thread 0's release
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(ctr), "r"(1u) : "memory");
        uint32_t spins = 0, ok = 1u;
        while (ld_acquire_gpu(ctr) < target) {
            if (++spins > kBarrierSpins) {
                atomicOr(err, kSortErrBit);
                ok = 0u;
                break;
            }
            __nanosleep(32);
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0u;
}

__global__ void __launch_bounds__(kOsThreads, 3) k_sort_coop(uint32_t* __restrict__ ka, int32_t* __restrict__ va,
                                                             uint32_t* __restrict__ kb, int32_t* __restrict__ vb,
                                                             const uint32_t* __restrict__ count, uint32_t n_max,
                                                             uint32_t* __restrict__ F, uint32_t* __restrict__ chunk_sum,
                                                             uint32_t* __restrict__ ctr, uint32_t* __restrict__ err) {
    // per-warp digit counts (then per-warp offsets); afterwards the tile's keys and values
    // in digit order (kOsTile each, the same 32 KB)
    __shared__ uint32_t s_cnt[kOsWarps * kRadix];
    __shared__ uint32_t s_local[kRadix]; // first tile-local position of each digit
    __shared__ uint32_t s_out[kRadix];   // the tile's digit counts, then its output positions
    __shared__ uint32_t s_cpre[kCoopMaxGrid];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_flag;
    const uint32_t n = min(*count, n_max);
    if (n == 0) return; // every block reads the same count: none waits at a barrier
    const uint32_t T = (n + kOsTile - 1) / kOsTile;
    // the grid is sized for the largest count; with fewer live tiles the blocks past them
    // leave at once (every block computes the same G), so they neither arrive at the
    // barriers nor hold a chunk of the scan
    const uint32_t G = min(gridDim.x, T);
    if (blockIdx.x >= G) return;
    const bool resident = T <= G; // at most one tile per block: it stays in shared memory
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const size_t L = (size_t)kRadix * T;
    const uint32_t chunk = (uint32_t)((L + G - 1) / G);
    uint32_t* s_key = s_cnt;
    int32_t* s_val = reinterpret_cast<int32_t*>(s_cnt + kOsTile);
    uint32_t barriers = 0;
    for (uint32_t pass = 0; pass < kRadixPasses; ++pass) {
        const uint32_t shift = kRadixBits * pass;
        uint32_t* kin = pass & 1u ? kb : ka;
        int32_t* vin = pass & 1u ? vb : va;
        uint32_t* kout = pass & 1u ? ka : kb;
        int32_t* vout = pass & 1u ? va : vb;
        // ---- A: rank every tile of this block ----
        for (uint32_t tile = blockIdx.x; tile < T; tile += G) {
            for (uint32_t i = threadIdx.x; i < kOsWarps * kRadix; i += kOsThreads) s_cnt[i] = 0u;
            __syncthreads();
            const uint32_t wbase = tile * kOsTile + w * kOsWarpKeys;
            uint32_t* wc = s_cnt + w * kRadix;
            uint32_t key[kOsRounds], pos[kOsRounds];
            int32_t val[kOsRounds];
#pragma unroll
            for (uint32_t r = 0; r < kOsRounds; ++r) {
                const uint32_t i = wbase + r * 32 + lane;
                key[r] = i < n ? __ldcg(kin + i) : 0u;
                val[r] = i < n ? __ldcg(vin + i) : 0;
            }
#pragma unroll
            for (uint32_t r = 0; r < kOsRounds; ++r) {
                const bool ok = wbase + r * 32 + lane < n;
                const uint32_t dig = (key[r] >> shift) & kRadixMask;
                uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
                for (uint32_t bit = 0; bit < kRadixBits; ++bit) {
                    const uint32_t b = __ballot_sync(0xffffffffu, (dig >> bit) & 1u);
                    peers &= ((dig >> bit) & 1u) ? b : ~b;
                }
                const uint32_t below = __popc(peers & ((1u << lane) - 1u));
                const uint32_t before = ok ? wc[dig] : 0u;
                __syncwarp();
                if (ok && below == 0u) wc[dig] = before + __popc(peers);
                __syncwarp();
                pos[r] = before + below;
            }
            __syncthreads();
            for (uint32_t d = threadIdx.x; d < kRadix; d += kOsThreads) {
                uint32_t acc = 0;
                for (uint32_t ww = 0; ww < kOsWarps; ++ww) {
                    const uint32_t c = s_cnt[ww * kRadix + d];
                    s_cnt[ww * kRadix + d] = acc;
                    acc += c;
                }
                s_out[d] = acc;
                F[(size_t)d * T + tile] = acc;
            }
            __syncthreads();
            {
                const uint32_t d0 = 4 * threadIdx.x;
                const uint32_t c0 = s_out[d0], c1 = s_out[d0 + 1], c2 = s_out[d0 + 2], c3 = s_out[d0 + 3];
                uint32_t tot;
                const uint32_t ex = block_excl_scan(c0 + c1 + c2 + c3, s_warp, tot);
                s_local[d0] = ex;
                s_local[d0 + 1] = ex + c0;
                s_local[d0 + 2] = ex + c0 + c1;
                s_local[d0 + 3] = ex + c0 + c1 + c2;
            }
            __syncthreads();
#pragma unroll
            for (uint32_t r = 0; r < kOsRounds; ++r) {
                if (wbase + r * 32 + lane < n) {
                    const uint32_t dig = (key[r] >> shift) & kRadixMask;
                    pos[r] += s_local[dig] + s_cnt[w * kRadix + dig];
                }
            }
            __syncthreads(); // the warp offsets are read: the same memory now stages the tile
#pragma unroll
            for (uint32_t r = 0; r < kOsRounds; ++r) {
                if (wbase + r * 32 + lane < n) {
                    s_key[pos[r]] = key[r];
                    s_val[pos[r]] = val[r];
                }
            }
            __syncthreads();
            if (!resident) { // back over the tile's own input range, in digit order
                const uint32_t tile_n = min(kOsTile, n - tile * kOsTile);
                for (uint32_t j = threadIdx.x; j < tile_n; j += kOsThreads) {
                    kin[tile * kOsTile + j] = s_key[j];
                    vin[tile * kOsTile + j] = s_val[j];
                }
                __syncthreads();
            }
        }
        if (!grid_barrier(ctr, ++barriers * G, err, &s_flag)) return;
        // ---- B: exclusive scan of F, one chunk per block ----
        {
            const size_t c0 = (size_t)blockIdx.x * chunk;
            const size_t c1 = min(L, c0 + chunk);
            const uint32_t per = (chunk + kOsThreads - 1) / kOsThreads;
            const size_t t0 = min(c1, c0 + (size_t)threadIdx.x * per);
            const size_t t1 = min(c1, t0 + per);
            uint32_t s = 0;
            for (size_t i = t0; i < t1; ++i) s += __ldcg(F + i);
            uint32_t tot;
            uint32_t run = block_excl_scan(s, s_warp, tot);
            for (size_t i = t0; i < t1; ++i) {
                const uint32_t v = __ldcg(F + i);
                F[i] = run;
                run += v;
            }
            if (threadIdx.x == 0) chunk_sum[blockIdx.x] = tot;
        }
        if (!grid_barrier(ctr, ++barriers * G, err, &s_flag)) return;
        // ---- C: output positions and the scatter ----
        // a block's only tile (the resident case) loads its scanned counts together with the
        // chunk sums: one round trip instead of two
        constexpr uint32_t Q = kRadix / kOsThreads;
        uint32_t fv[Q];
        if (resident && blockIdx.x < T) {
#pragma unroll
            for (uint32_t q = 0; q < Q; ++q) fv[q] = __ldcg(F + (size_t)(threadIdx.x + q * kOsThreads) * T + blockIdx.x);
        }
        {   // exclusive prefix of the chunk sums; thread t owns chunks 4t..4t+3
            const uint32_t q0 = 4 * threadIdx.x;
            uint32_t c[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) c[k] = q0 + k < G ? __ldcg(chunk_sum + q0 + k) : 0u;
            uint32_t tot;
            const uint32_t ex = block_excl_scan(c[0] + c[1] + c[2] + c[3], s_warp, tot);
            uint32_t acc = ex;
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                if (q0 + k < kCoopMaxGrid) s_cpre[q0 + k] = acc;
                acc += c[k];
            }
        }
        __syncthreads();
        for (uint32_t tile = blockIdx.x; tile < T; tile += G) {
            const uint32_t tile_n = min(kOsTile, n - tile * kOsTile);
            if (!resident) {
                for (uint32_t j = threadIdx.x; j < tile_n; j += kOsThreads) {
                    s_key[j] = __ldcg(kin + tile * kOsTile + j);
                    s_val[j] = __ldcg(vin + tile * kOsTile + j);
                }
                __syncthreads();
                // first tile-local position of each digit present in the tile
                for (uint32_t j = threadIdx.x; j < tile_n; j += kOsThreads) {
                    const uint32_t d = (s_key[j] >> shift) & kRadixMask;
                    if (j == 0 || ((s_key[j - 1] >> shift) & kRadixMask) != d) s_local[d] = j;
                }
            }
#pragma unroll
            for (uint32_t q = 0; q < Q; ++q) {
                const uint32_t d = threadIdx.x + q * kOsThreads;
                const size_t idx = (size_t)d * T + tile;
                s_out[d] = (resident ? fv[q] : __ldcg(F + idx)) + s_cpre[idx / chunk];
            }
            __syncthreads();
            for (uint32_t j = threadIdx.x; j < tile_n; j += kOsThreads) {
                const uint32_t k = s_key[j];
                const uint32_t d = (k >> shift) & kRadixMask;
                const uint32_t dst = s_out[d] + (j - s_local[d]);
                if (dst < n) {
                    kout[dst] = k;
                    vout[dst] = s_val[j];
                } else {
                    atomicOr(err, kSortErrBit);
                }
            }
            __syncthreads(); // shared memory is reused by the next tile or pass
        }
        if (pass + 1 < kRadixPasses && !grid_barrier(ctr, ++barriers * G, err, &s_flag)) return;
    }
}

// ------------------------------------------------------------------------------------
// End of a pass, one thread per slot: a path still alive after its last secondary ray
// only adds the environment or the emission where that ray ended (no group logic is left
// to do), then the sample's radiance goes to its pixel.  Each pixel has one slot per pass
// and passes run in sample order, so the sum keeps that order.  With p.accum_mode, a job's
// first sample starts the sum (no cleared buffer is read) and its last sample writes the
// output, sum / spp, instead of the sum.
__global__ void k_finish_accumulate(PassArgs p, const int32_t* __restrict__ pixel,
                                    const uint16_t* __restrict__ slot_job, const uint8_t* __restrict__ alive,
                                    const int2* __restrict__ hit, const float4* __restrict__ ray_o,
                                    const float4* __restrict__ ray_d, const float4* __restrict__ beta,
                                    const float4* __restrict__ radiance, uint32_t n_slots,
                                    float4* __restrict__ accum, cr_debug dbg, uint32_t dbg_npx) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n_slots) return;
    uint32_t s = u;
    if (p.rolling) { // the slots of the jobs that end a sample now, from the launch lists
        const uint32_t e = launch_entry(p.launch_prefix, p.n_launch, u);
        s = p.jobs[p.launch_job[e]].slot_tile * p.m + (u - p.launch_prefix[e]);
    }
    const int pix = pixel[s];
    if (pix < 0) return;
    const JobDev& J = p.jobs[slot_job[s]];
    const bool on = alive[s] != 0;
    const float4 r4 = radiance[s];
    float3 L = make_float3(r4.x, r4.y, r4.z);
    if (on) {
        const SceneDev& sc = p.scenes[J.scene];
        const int2 h = hit[s];
        const float4 bt = beta[s];
        if (dbg.prim)
            dbg.prim[(p.bounce - 1) * dbg_npx + (uint32_t)pix] =
                h.x >= 0 ? __float_as_int(__ldg(&sc.tris[3 * h.x]).w) : -1;
        if (dbg.ray) capture_trace(dbg, (p.bounce - 1) * dbg_npx + (uint32_t)pix, ray_o[s], ray_d[s], h, bt);
        bool ok = h.x >= 0;
        CR_DBG(ok = ok && dbg_in_range(&sc, (uint32_t)h.x, kDbgHit, sc.n_tris) &&
                    dbg_in_range(&sc, (uint32_t)__float_as_int(__ldg(&sc.tris[3 * h.x + 1]).w), kDbgMat, sc.n_mats);)
        if (h.x < 0) {
            add_environment(sc, bt, L);
        } else if (ok) {
            const float4 v1 = __ldg(&sc.tris[3 * h.x + 1]);
            const int mat = __float_as_int(v1.w);
            const float4 m0 = __ldg(&sc.mats[2 * mat + 0]);
            if ((uint32_t)__float_as_int(m0.x) == kMatEmitter) {
                const float4 v0 = __ldg(&sc.tris[3 * h.x + 0]);
                const float4 v2 = __ldg(&sc.tris[3 * h.x + 2]);
                const float4 m1 = __ldg(&sc.mats[2 * mat + 1]);
                add_emission(sc, v0, v1, v2, m1, bt, h, ray_d[s], J.nee != 0, L);
            }
        }
    }
    const uint32_t at = J.px_base + (uint32_t)pix;
    const bool first = (p.accum_mode & 1u) && (J.sample_flags & 1u);
    const bool last = (p.accum_mode & 2u) && (J.sample_flags & 2u);
    float4 a = first ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : accum[at];
    a.x += L.x;
    a.y += L.y;
    a.z += L.z;
    if (last) {
        J.out[3 * pix + 0] = a.x * J.inv_spp;
        J.out[3 * pix + 1] = a.y * J.inv_spp;
        J.out[3 * pix + 2] = a.z * J.inv_spp;
    } else {
        accum[at] = a;
    }
}

// Job of an accumulation pixel: the last job whose first pixel is <= i.
__device__ __forceinline__ uint32_t job_of_pixel(const JobDev* jobs, uint32_t n_jobs, uint32_t i) {
    uint32_t lo = 0, hi = n_jobs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (jobs[mid].px_base <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void k_output(const JobDev* __restrict__ jobs, uint32_t n_jobs, const float4* __restrict__ accum,
                         uint32_t npx_total) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npx_total) return;
    const JobDev& J = jobs[job_of_pixel(jobs, n_jobs, i)];
    const uint32_t p = i - J.px_base;
    const float4 a = accum[i];
    J.out[3 * p + 0] = a.x * J.inv_spp;
    J.out[3 * p + 1] = a.y * J.inv_spp;
    J.out[3 * p + 2] = a.z * J.inv_spp;
}

__global__ void k_output_one(const float4* __restrict__ accum, uint32_t npx, float inv_spp, float* __restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    const float4 a = accum[i];
    out[3 * i + 0] = a.x * inv_spp;
    out[3 * i + 1] = a.y * inv_spp;
    out[3 * i + 2] = a.z * inv_spp;
}

__global__ void k_philox(uint64_t seed, const uint32_t* __restrict__ ctr, uint32_t n, uint32_t* __restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 r = philox_seed(seed, ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    out[4 * i + 0] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

__global__ void k_sample(uint32_t kind, uint32_t n, const float* __restrict__ wo, const float* __restrict__ u,
                         const float* __restrict__ param, float* __restrict__ wi, float* __restrict__ weight,
                         uint8_t* __restrict__ valid) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V3 r = v3(0.0f, 0.0f, 0.0f);
    float w[3] = {0.0f, 0.0f, 0.0f};
    bool ok = true;
    if (kind == 0) {
        r = sample_cosine(u[2 * i], u[2 * i + 1]);
        w[0] = w[1] = w[2] = 1.0f;
    } else if (kind == 1) {
        const float f0[3] = {param[4 * i + 1], param[4 * i + 2], param[4 * i + 3]};
        ok = sample_ggx(v3(wo[3 * i], wo[3 * i + 1], wo[3 * i + 2]), param[4 * i], f0, u[2 * i], u[2 * i + 1], r, w);
    } else if (kind == 2) {
        r = v3(-wo[3 * i], -wo[3 * i + 1], wo[3 * i + 2]);
        w[0] = w[1] = w[2] = 1.0f;
        ok = wo[3 * i + 2] > 0.0f;
    } else {
        float s, c;
        sincos_poly(u[2 * i], s, c);
        r = v3(s, c, 0.0f);
    }
    wi[3 * i + 0] = r.x;
    wi[3 * i + 1] = r.y;
    wi[3 * i + 2] = r.z;
    weight[3 * i + 0] = w[0];
    weight[3 * i + 1] = w[1];
    weight[3 * i + 2] = w[2];
    valid[i] = ok ? 1 : 0;
}

} // namespace

// ------------------------------------------------------------------------------------
// Launchers.
void launch_raygen(const PassArgs& p, PathBuffers& b, cudaStream_t st, LaunchCount& lc) {
    const uint32_t block = p.m > 256 ? p.m : 256;
    const uint32_t tiles_per_block = block / p.m;
    const uint32_t grid = (p.n_tiles + tiles_per_block - 1) / tiles_per_block;
#ifndef CR_PRIMARY_PIXEL_ORDER
#define CR_PRIMARY_PIXEL_ORDER 1
#endif
    // the ray queue is free until the first compaction: it carries the primary trace's order
    k_raygen<<<grid, block, block * sizeof(uint16_t), st>>>(p, b.pixel, b.slot_job, b.slot_scene, b.ray_o, b.ray_d,
                                                             b.beta, b.radiance, b.alive,
                                                             CR_PRIMARY_PIXEL_ORDER ? b.ray_queue : nullptr,
                                                             b.counts + 8);
    lc.n++;
}

bool primary_pixel_order() { return CR_PRIMARY_PIXEL_ORDER != 0; }

void launch_groups(const CamBasis& cam, uint32_t tile_w, uint32_t tile_h, uint32_t interleave, uint64_t seed,
                   uint32_t frame, uint32_t* slot_of_pixel, cudaStream_t st, LaunchCount& lc) {
    const uint32_t npx = cam.width * cam.height;
    k_groups<<<(npx + 255) / 256, 256, 0, st>>>(cam, tile_w, tile_h, interleave, seed, frame, slot_of_pixel);
    lc.n++;
}

static ShadeArgs shade_args(const PassArgs& p, PathBuffers& b, bool first, bool compact, const cr_debug* dbg) {
    ShadeArgs a;
    a.jobs = p.jobs;
    a.scenes = p.scenes;
    a.slot_job = b.slot_job;
    a.pixel = b.pixel;
    a.ray_o = b.ray_o;
    a.ray_d = b.ray_d;
    a.hit = b.hit;
    a.beta = b.beta;
    a.radiance = b.radiance;
    a.alive = b.alive;
    // group queue written by the previous shade's compaction (double-buffered)
    a.group_queue = first ? nullptr : b.group_queue + (size_t)((p.bounce - 1) & 1) * b.n_groups;
    a.group_count = first ? nullptr : b.counts + 8 + 2 * (p.bounce - 1) + 1;
    a.n_groups_max = b.n_groups;
    if (dbg) a.dbg = *dbg;
    else a.dbg = cr_debug{};
    a.npx = p.npx;
    const bool nee = p.nee && b.shadow_d;
    a.shadow_o = nee ? b.shadow_o : nullptr;
    a.shadow_d = nee ? b.shadow_d : nullptr;
    a.shadow_c = nee ? b.shadow_c : nullptr;
    a.ray_queue = compact ? b.ray_queue : nullptr;
    a.group_queue_out = b.group_queue + (size_t)(p.bounce & 1) * b.n_groups;
    a.queue_counts = b.counts + 8 + 2 * p.bounce;
    a.rays_queued = reinterpret_cast<unsigned long long*>(b.counts + kStatWord) + p.bounce;
    a.queue_err = b.counts + kQueueErrWord;
    a.ray_cap = b.n_groups * p.k;
    a.group_cap = b.n_groups;
    return a;
}

void launch_shadow(const PassArgs& p, PathBuffers& b, bool first, bool bvh8, cudaStream_t st, LaunchCount& lc) {
    if (!p.nee || !b.shadow_d) return;
    const ShadeArgs a = shade_args(p, b, first, false, nullptr);
    launch_shadow_rays(p.scenes, b.slot_scene, b.shadow_o, b.shadow_d, b.shadow_c, a.group_queue, a.group_count,
                       a.n_groups_max, p.k, b.radiance, reinterpret_cast<unsigned long long*>(b.counts + kShadowWord),
                       bvh8, st, lc);
}

void launch_shade(const PassArgs& p, PathBuffers& b, bool first, bool compact, const cr_debug* dbg,
                  cudaStream_t st, LaunchCount& lc) {
    ShadeArgs a = shade_args(p, b, first, compact, dbg);
    const uint32_t n_pos = b.n_groups * p.k;
    if (p.k <= 32) {
        k_shade_warp<<<(n_pos + CR_SHADE_WARP_BLOCK - 1) / CR_SHADE_WARP_BLOCK, CR_SHADE_WARP_BLOCK, 0, st>>>(a, p);
    } else {
        k_shade_block<<<(n_pos + 255) / 256, 256, 0, st>>>(a, p);
    }
    lc.n++;
}

// Rolling wavefront.  Queue words: pair q = counts + 8 + 2 q holds (rays, groups) appended
// for the iteration that reads group queue q; the caller zeroes the pair an iteration appends
// to before its first launch.
void launch_raygen_rolling(const PassArgs& p, PathBuffers& b, uint32_t n_tiles, cudaStream_t st, LaunchCount& lc) {
    if (!n_tiles) return;
    PassArgs q = p;
    q.n_tiles = n_tiles;
    const uint32_t block = p.m > 256 ? p.m : 256;
    const uint32_t tiles_per_block = block / p.m;
    const uint32_t grid = (n_tiles + tiles_per_block - 1) / tiles_per_block;
    // shared memory: the inverse shuffle (2 B per thread), then one live flag per group
    k_raygen<<<grid, block, block * (sizeof(uint16_t) + sizeof(uint32_t)) + 4, st>>>(
        q, b.pixel, b.slot_job, b.slot_scene, b.ray_o, b.ray_d, b.beta, b.radiance, b.alive, nullptr, nullptr);
    lc.n++;
}

static ShadeArgs shade_args_rolling(const PassArgs& p, PathBuffers& b, uint32_t parity, uint32_t n_groups_max) {
    ShadeArgs a = shade_args(p, b, false, true, nullptr);
    a.group_queue = b.group_queue + (size_t)parity * b.n_groups;
    a.group_count = b.counts + 8 + 2 * parity + 1;
    a.n_groups_max = n_groups_max;
    a.group_queue_out = b.group_queue + (size_t)(parity ^ 1u) * b.n_groups;
    a.queue_counts = b.counts + 8 + 2 * (parity ^ 1u);
    a.rays_queued = reinterpret_cast<unsigned long long*>(b.counts + kStatWord) + 1;
    a.ray_cap = b.n_groups * p.k;
    a.group_cap = b.n_groups;
    return a;
}

void launch_shade_rolling(const PassArgs& p, PathBuffers& b, uint32_t parity, uint32_t n_groups_max,
                          cudaStream_t st, LaunchCount& lc) {
    if (!n_groups_max) return;
    ShadeArgs a = shade_args_rolling(p, b, parity, n_groups_max);
    const uint32_t n_pos = n_groups_max * p.k;
    if (p.k <= 32) {
        k_shade_warp<<<(n_pos + CR_SHADE_WARP_BLOCK - 1) / CR_SHADE_WARP_BLOCK, CR_SHADE_WARP_BLOCK, 0, st>>>(a, p);
    } else {
        k_shade_block<<<(n_pos + 255) / 256, 256, 0, st>>>(a, p);
    }
    lc.n++;
}

void launch_shadow_rolling(const PassArgs& p, PathBuffers& b, uint32_t parity, uint32_t n_groups_max, bool bvh8,
                           cudaStream_t st, LaunchCount& lc) {
    if (!p.nee || !b.shadow_d || !n_groups_max) return;
    const ShadeArgs a = shade_args_rolling(p, b, parity, n_groups_max);
    launch_shadow_rays(p.scenes, b.slot_scene, b.shadow_o, b.shadow_d, b.shadow_c, a.group_queue, a.group_count,
                       n_groups_max, p.k, b.radiance, reinterpret_cast<unsigned long long*>(b.counts + kShadowWord),
                       bvh8, st, lc);
}

void launch_finish_rolling(const PassArgs& p, PathBuffers& b, uint32_t n_slots, cudaStream_t st, LaunchCount& lc) {
    if (!n_slots) return;
    k_finish_accumulate<<<(n_slots + 255) / 256, 256, 0, st>>>(p, b.pixel, b.slot_job, b.alive, b.hit, b.ray_o,
                                                               b.ray_d, b.beta, b.radiance, n_slots, b.accum,
                                                               cr_debug{}, 0);
    lc.n++;
}

void launch_compact(const PassArgs& p, PathBuffers& b, bool first, cudaStream_t st, LaunchCount& lc) {
    const uint32_t K = p.k;
    const uint32_t n_pos = b.n_groups * K;
    const uint32_t n_blocks = (n_pos + kCompactBlock - 1) / kCompactBlock;
    const int32_t* gq_in = first ? nullptr : b.group_queue + (size_t)((p.bounce - 1) & 1) * b.n_groups;
    const uint32_t* ng_in = first ? nullptr : b.counts + 8 + 2 * (p.bounce - 1) + 1;
    int32_t* gq_out = b.group_queue + (size_t)(p.bounce & 1) * b.n_groups;
    uint32_t* out_counts = b.counts + 8 + 2 * p.bounce;
    k_compact_count<<<n_blocks, kCompactBlock, 0, st>>>(gq_in, ng_in, b.n_groups, K, b.alive, b.block_counts);
    k_compact_scan<<<1, 1024, 0, st>>>(b.block_counts, n_blocks, out_counts,
                                      reinterpret_cast<unsigned long long*>(b.counts + kStatWord) + p.bounce);
    k_compact_scatter<<<n_blocks, kCompactBlock, 0, st>>>(gq_in, ng_in, b.n_groups, K, b.alive, b.block_counts,
                                                         b.ray_queue, gq_out);
    lc.n += 3;
}

void launch_finish_accumulate(const PassArgs& p, PathBuffers& b, const cr_debug* dbg, cudaStream_t st,
                              LaunchCount& lc) {
    const uint32_t n_slots = p.n_tiles * p.m;
    k_finish_accumulate<<<(n_slots + 255) / 256, 256, 0, st>>>(p, b.pixel, b.slot_job, b.alive, b.hit, b.ray_o,
                                                               b.ray_d, b.beta, b.radiance, n_slots, b.accum,
                                                               dbg ? *dbg : cr_debug{}, p.npx);
    lc.n++;
}

void launch_output(const JobDev* jobs, uint32_t n_jobs, const float4* accum, uint32_t npx_total, cudaStream_t st,
                   LaunchCount& lc) {
    k_output<<<(npx_total + 255) / 256, 256, 0, st>>>(jobs, n_jobs, accum, npx_total);
    lc.n++;
}

void launch_output_one(const float4* accum, uint32_t npx, float inv_spp, float* out, cudaStream_t st, LaunchCount& lc) {
    if (!npx) return;
    k_output_one<<<(npx + 255) / 256, 256, 0, st>>>(accum, npx, inv_spp, out);
    lc.n++;
}

void launch_philox(uint64_t seed, const uint32_t* ctr, uint32_t n, uint32_t* out, cudaStream_t st, LaunchCount& lc) {
    if (!n) return;
    k_philox<<<(n + 255) / 256, 256, 0, st>>>(seed, ctr, n, out);
    lc.n++;
}

void launch_sample(uint32_t kind, uint32_t n, const float* wo, const float* u, const float* param, float* wi,
                   float* weight, uint8_t* valid, cudaStream_t st, LaunchCount& lc) {
    if (!n) return;
    k_sample<<<(n + 255) / 256, 256, 0, st>>>(kind, n, wo, u, param, wi, weight, valid);
    lc.n++;
}

// SMs of the current device (grids of a fixed number of blocks per SM).
static int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached[dev] = v;
    }
    return cached[dev];
}

// Resident k_sort_coop blocks per SM: its grid is one wave, every block resident at once.
static uint32_t sort_blocks_per_sm() {
    static int cached = 0;
    if (!cached) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sort_coop, kOsThreads, 0) != cudaSuccess || nb <= 0)
            nb = 1;
        cached = nb;
    }
    return (uint32_t)cached;
}

// The three radix passes over keys/values (ka, va) -> (kb, vb) -> (ka, va) -> (kb, vb) as one
// cooperative launch; ws is the sort workspace (digit counts and the barrier counter
// cleared, then F and the chunk sums).
static void launch_radix_passes(uint32_t* ka, int32_t* va, uint32_t* kb, int32_t* vb, const uint32_t* count,
                                uint32_t n_max, uint32_t* ws, uint32_t* err, cudaStream_t st, LaunchCount& lc) {
    const uint32_t tiles_max = (n_max + kOsTile - 1) / kOsTile;
    const size_t stride = (size_t)tiles_max * kRadix;
    const uint32_t grid = max(1u, min(min(tiles_max, kCoopMaxGrid), sort_blocks_per_sm() * (uint32_t)sm_count()));
    uint32_t* F = ws + kSortF;
    uint32_t* chunk_sum = ws + kSortF + stride;
    uint32_t* ctr = ws + kSortCtr;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kOsThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_sort_coop, ka, va, kb, vb, count, n_max, F, chunk_sum, ctr, err);
    lc.n++;
}

// Sort the current bounce's ray queue by its reordering key; returns the sorted slot queue.
const int32_t* launch_morton_sort(const PassArgs& p, PathBuffers& b, uint32_t bounce, uint32_t key_kind,
                                  cudaStream_t st, LaunchCount& lc) {
    const uint32_t n_max = b.n_slots;
    const uint32_t* count = b.counts + 8 + 2 * bounce;
    uint32_t* ws = b.sort_hist;
    // one thread per key: every queue entry's ray gather is in flight at once
    k_morton<<<(n_max + 511) / 512, 512, 0, st>>>(b.ray_o, b.ray_d, b.ray_queue, count, n_max, p.scenes, b.slot_scene,
                                                 key_kind, b.keys, b.vals, b.vals + n_max, ws + kSortCtr);
    lc.n++;
    launch_radix_passes(b.keys, b.vals, b.keys + n_max, b.vals + n_max, count, n_max, ws, b.counts + kQueueErrWord,
                        st, lc);
    return b.vals + n_max; // the last pass's output
}

// The ray sort on a caller's n keys (low 30 bits) and values, in buffers of the sort's
// layout: keys[0, 2n) and vals[0, 2n), ws of sort_hist_len(n) words; returns the sorted
// values (the sorted keys are at the same offset of keys).  Used by cr_debug_sort.
int32_t* launch_sort_only(const uint32_t* key_in, const int32_t* val_in, uint32_t n, uint32_t* keys, int32_t* vals,
                          uint32_t* ws, uint32_t* count, uint32_t* err, cudaStream_t st, LaunchCount& lc) {
    k_morton<<<(n + 511) / 512, 512, 0, st>>>(nullptr, nullptr, reinterpret_cast<const int32_t*>(key_in),
                                                             count, n, nullptr,
                                                             reinterpret_cast<const uint16_t*>(val_in), 0, keys, vals,
                                                             vals + n, ws + kSortCtr);
    lc.n++;
    launch_radix_passes(keys, vals, keys + n, vals + n, count, n, ws, err, st, lc);
    return vals + n;
}

void launch_scan_counts(uint32_t* block_counts, uint32_t n_blocks, uint32_t* total, cudaStream_t st) {
    // k_compact_scan scans both columns; column 1 is zero here and its total lands in total[1]
    k_compact_scan<<<1, 1024, 0, st>>>(block_counts, n_blocks, total, nullptr);
}

// words of the sort workspace: the barrier counter, the digit counts of every tile, the chunk sums
uint32_t sort_hist_len(uint32_t n_slots) {
    return kSortF + ((n_slots + kOsTile - 1) / kOsTile) * kRadix + kCoopMaxGrid;
}
uint32_t compact_blocks(uint32_t n_pos) { return (n_pos + kCompactBlock - 1) / kCompactBlock; }

} // namespace cr
