// cr_api.cpp -- the C ABI of libcr.so (include/cr.h): argument checking, scene upload,
// render orchestration of the wavefront stages on one stream, and the parity entry points.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include "cr_internal.h"

namespace cr {
namespace {

thread_local std::string g_err;

cr_status fail(cr_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CR_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            cr_status s_ = e_ == cudaErrorMemoryAllocation ? CR_ERR_OOM : CR_ERR_CUDA;    \
            return fail(s_, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                 \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device allocation released on scope exit unless kept.
struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    ~DevMem() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = n;
        return cudaMalloc(&p, n ? n : 16);
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

} // namespace

CamBasis make_camera(const cr_camera& c) {
    double p[3] = {c.pos[0], c.pos[1], c.pos[2]};
    double la[3] = {c.look_at[0], c.look_at[1], c.look_at[2]};
    double up[3] = {c.up[0], c.up[1], c.up[2]};
    double f[3] = {la[0] - p[0], la[1] - p[1], la[2] - p[2]};
    auto norm = [](double* a) {
        double l = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        a[0] /= l;
        a[1] /= l;
        a[2] /= l;
    };
    auto cross = [](const double* a, const double* b, double* r) {
        r[0] = a[1] * b[2] - a[2] * b[1];
        r[1] = a[2] * b[0] - a[0] * b[2];
        r[2] = a[0] * b[1] - a[1] * b[0];
    };
    norm(f);
    double r[3], u[3];
    cross(f, up, r);
    norm(r);
    cross(r, f, u);
    const double th = std::tan(c.vfov_deg * (3.14159265358979323846 / 180.0) * 0.5);
    CamBasis b;
    for (int k = 0; k < 3; ++k) {
        b.pos[k] = c.pos[k];
        b.fwd[k] = (float)f[k];
        b.right[k] = (float)r[k];
        b.up[k] = (float)u[k];
    }
    b.ty = (float)th;
    b.tx = (float)(th * ((double)c.width / (double)c.height));
    b.width = c.width;
    b.height = c.height;
    return b;
}

} // namespace cr

// ------------------------------------------------------------------------------------
struct cr_scene {
    cr::DevScene dev;
    cr_scene_info info;
    void* d_nodes2 = nullptr;
    void* d_nodes8 = nullptr;
    void* d_nodes4 = nullptr;
    void* d_tris = nullptr;
    void* d_tris8 = nullptr;
    void* d_mats = nullptr;
    void* d_lights = nullptr; // emitter records and their running areas (one allocation)
    cr::SceneDev* d_entries = nullptr; // [0] BVH2 layout, [1] BVH8-Q layout (scene-table entries)
    int device = -1;                   // the CUDA device the scene's memory lives on
    // render workspace and job tables, grown on demand
    cr::Workspace ws;
    cr::Plan plan_dev;
    float* d_out = nullptr;
    size_t out_cap = 0;
};

using namespace cr;

namespace cr {
void set_last_error(const char* msg) { g_err = msg; }
const DevScene* dev_scene_of(const cr_scene* s) { return &s->dev; }
const SceneDev* dev_scene_entry(const cr_scene* s, bool bvh8) { return s->d_entries + (bvh8 ? 1 : 0); }
bool scene_has_bvh8(const cr_scene* s) { return s->dev.nodes8 != nullptr; }
int scene_device(const cr_scene* s) { return s->device; }
} // namespace cr

extern "C" const char* cr_last_error(void) { return g_err.c_str(); }
#ifndef CR_DEBUG
#define CR_DEBUG 0
#endif
extern "C" const char* cr_version(void) { return CR_DEBUG ? "cr 0.1 sm_103a debug" : "cr 0.1 sm_103a"; }

namespace cr {
// A debug build's finding on a scene after a synchronised call: CR_OK, or CR_ERR_CUDA when a
// kernel found a node, triangle or material index out of range (the word is then cleared).
static cr_status debug_word_status(const cr_scene* s) {
#if CR_DEBUG
    uint32_t w = 0;
    if (cudaMemcpy(&w, s->dev.err, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(CR_ERR_CUDA, "debug build: reading the error word failed");
    if (w) {
        cudaMemset(s->dev.err, 0, 4);
        return fail(CR_ERR_CUDA, "debug build: index checks failed (bits 0x%x: 1 node, 2 triangle, 4 hit, 8 material)",
                    w);
    }
#else
    (void)s;
#endif
    return CR_OK;
}
} // namespace cr

extern "C" cr_status cr_scene_create(const float* tri_xyz, uint32_t n_tri, const uint32_t* tri_mat,
                                     const cr_material* mats, uint32_t n_mat, const cr_env* env, uint32_t bvh_flags,
                                     cr_scene** out) {
    g_err.clear();
    if (!out) return fail(CR_ERR_INVALID_ARG, "cr_scene_create: out is NULL");
    *out = nullptr;
    if (!tri_xyz || !tri_mat || !mats) return fail(CR_ERR_INVALID_ARG, "cr_scene_create: NULL array");
    if (n_tri == 0 || n_tri > (1u << 28)) return fail(CR_ERR_INVALID_ARG, "cr_scene_create: n_tri=%u out of range", n_tri);
    if (n_mat == 0) return fail(CR_ERR_INVALID_ARG, "cr_scene_create: n_mat is 0");
    if (bvh_flags & ~(uint32_t)(CR_BVH2 | CR_BVH8Q | CR_BVH4))
        return fail(CR_ERR_INVALID_ARG, "cr_scene_create: bad bvh_flags");
    for (size_t i = 0; i < 9 * (size_t)n_tri; ++i)
        if (!std::isfinite(tri_xyz[i]))
            return fail(CR_ERR_INVALID_ARG, "cr_scene_create: vertex coordinate %zu of triangle %zu is not finite", i % 9,
                        i / 9);
    for (uint32_t t = 0; t < n_tri; ++t)
        if (tri_mat[t] >= n_mat)
            return fail(CR_ERR_INVALID_ARG, "cr_scene_create: triangle %u uses material %u >= n_mat %u", t, tri_mat[t], n_mat);
    for (uint32_t m = 0; m < n_mat; ++m) {
        if (mats[m].type > CR_MAT_TRANSLUCENT)
            return fail(CR_ERR_INVALID_ARG, "cr_scene_create: material %u type %u", m, mats[m].type);
        if (mats[m].type == CR_MAT_DIELECTRIC && !(mats[m].roughness > 0.0f && mats[m].roughness <= 10.0f))
            return fail(CR_ERR_INVALID_ARG, "cr_scene_create: material %u index of refraction %g not in (0, 10]", m,
                        mats[m].roughness);
        if (mats[m].type == CR_MAT_GGX && !(mats[m].roughness > 0.0f && mats[m].roughness <= 1.0f))
            return fail(CR_ERR_INVALID_ARG, "cr_scene_create: material %u roughness %g not in (0, 1]", m, mats[m].roughness);
    }
    std::unique_ptr<cr_scene> s(new (std::nothrow) cr_scene());
    if (!s) return fail(CR_ERR_OOM, "cr_scene_create: host allocation");
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(CR_ERR_CUDA, "cr_scene_create: no CUDA device");
    }
    const auto t0 = std::chrono::steady_clock::now();
    const unsigned hc = std::thread::hardware_concurrency();
    HostBVH2 b2;
    try {
        b2 = build_bvh2(tri_xyz, n_tri, hc ? (int)hc : 4);
    } catch (const std::bad_alloc&) {
        return fail(CR_ERR_OOM, "cr_scene_create: host allocation during BVH build");
    }
    if (b2.depth >= kBvh2StackCapacity)
        return fail(CR_ERR_STACK_OVERFLOW, "cr_scene_create: BVH2 depth %u needs a deeper traversal stack (%u)", b2.depth,
                    kBvh2StackCapacity);
    // triangles in leaf order: v0 | original index, v1 | material, v2 | 0
    std::vector<float> tris(12 * (size_t)n_tri);
    for (uint32_t i = 0; i < n_tri; ++i) {
        const uint32_t t = b2.leaf_order[i];
        float* o = &tris[12 * (size_t)i];
        for (int v = 0; v < 3; ++v)
            for (int k = 0; k < 3; ++k) o[4 * v + k] = tri_xyz[9 * (size_t)t + 3 * v + k];
        int32_t orig = (int32_t)t, mat = (int32_t)tri_mat[t];
        std::memcpy(&o[3], &orig, 4);
        std::memcpy(&o[7], &mat, 4);
        o[11] = 0.0f;
    }
    HostBVH8 b8;
    std::vector<float> tris8;
    if (bvh_flags & CR_BVH8Q) {
        try {
            b8 = build_bvh8q(b2, tri_xyz);
        } catch (const std::bad_alloc&) {
            return fail(CR_ERR_OOM, "cr_scene_create: host allocation during BVH8-Q build");
        }
        if (b8.stack_bound > kBvh8StackCapacity)
            return fail(CR_ERR_STACK_OVERFLOW, "cr_scene_create: BVH8-Q needs a %u-entry stack (> %u)", b8.stack_bound,
                        kBvh8StackCapacity);
        tris8.resize(12 * b8.leaf_order.size());
        for (size_t i = 0; i < b8.leaf_order.size(); ++i) {
            const uint32_t t = b8.leaf_order[i];
            float* o = &tris8[12 * i];
            for (int v = 0; v < 3; ++v)
                for (int k = 0; k < 3; ++k) o[4 * v + k] = tri_xyz[9 * (size_t)t + 3 * v + k];
            int32_t orig = (int32_t)t, mat = (int32_t)tri_mat[t];
            std::memcpy(&o[3], &orig, 4);
            std::memcpy(&o[7], &mat, 4);
            o[11] = 0.0f;
        }
    }
    HostBVH4 b4;
    if (bvh_flags & CR_BVH4) {
        try {
            b4 = build_bvh4(b2);
        } catch (const std::bad_alloc&) {
            return fail(CR_ERR_OOM, "cr_scene_create: host allocation during BVH4 build");
        }
        if (b4.stack_bound > kBvh4StackCapacity)
            return fail(CR_ERR_STACK_OVERFLOW, "cr_scene_create: BVH4 needs a %u-entry stack (> %u)", b4.stack_bound,
                        kBvh4StackCapacity);
    }
    std::vector<float> mt(8 * (size_t)n_mat);
    for (uint32_t m = 0; m < n_mat; ++m) {
        int32_t ty = (int32_t)mats[m].type;
        std::memcpy(&mt[8 * m], &ty, 4);
        mt[8 * m + 1] = mats[m].albedo[0];
        mt[8 * m + 2] = mats[m].albedo[1];
        mt[8 * m + 3] = mats[m].albedo[2];
        mt[8 * m + 4] = mats[m].roughness;
        mt[8 * m + 5] = mats[m].emission[0];
        mt[8 * m + 6] = mats[m].emission[1];
        mt[8 * m + 7] = mats[m].emission[2];
    }
    // Emitter table for next-event estimation: triangle-index order, 4 float4 per emitter
    // (v0|orig, v1, v2, emission) and the float running sum of the areas, each area
    // 0.5 |(v1 - v0) x (v2 - v0)| evaluated in double.
    std::vector<float> lrec, lcdf;
    {
        double run = 0.0;
        for (uint32_t t = 0; t < n_tri; ++t) {
            const cr_material& mm = mats[tri_mat[t]];
            if (mm.type != CR_MAT_EMITTER) continue;
            const float* v = &tri_xyz[9 * (size_t)t];
            double e1[3], e2[3];
            for (int k = 0; k < 3; ++k) {
                e1[k] = (double)v[3 + k] - (double)v[k];
                e2[k] = (double)v[6 + k] - (double)v[k];
            }
            const double cx = e1[1] * e2[2] - e1[2] * e2[1];
            const double cy = e1[2] * e2[0] - e1[0] * e2[2];
            const double cz = e1[0] * e2[1] - e1[1] * e2[0];
            run += 0.5 * std::sqrt((cx * cx + cy * cy) + cz * cz);
            lcdf.push_back((float)run);
            int32_t orig = (int32_t)t;
            float ob;
            std::memcpy(&ob, &orig, 4);
            const float rec[16] = {v[0], v[1], v[2], ob, v[3], v[4], v[5], 0.0f, v[6], v[7], v[8], 0.0f,
                                   mm.emission[0], mm.emission[1], mm.emission[2], 0.0f};
            lrec.insert(lrec.end(), rec, rec + 16);
        }
    }
    const auto t1 = std::chrono::steady_clock::now();
    DevMem dn, dt, dm;
    CR_CUDA(dn.alloc(b2.nodes.size() * sizeof(float)));
    CR_CUDA(dt.alloc(tris.size() * sizeof(float)));
    CR_CUDA(dm.alloc(mt.size() * sizeof(float)));
    CR_CUDA(cudaMemcpy(dn.p, b2.nodes.data(), dn.bytes, cudaMemcpyHostToDevice));
    CR_CUDA(cudaMemcpy(dt.p, tris.data(), dt.bytes, cudaMemcpyHostToDevice));
    CR_CUDA(cudaMemcpy(dm.p, mt.data(), dm.bytes, cudaMemcpyHostToDevice));
    DevMem dn8, dt8;
    if (bvh_flags & CR_BVH8Q) {
        CR_CUDA(dn8.alloc(b8.nodes.size() * sizeof(uint32_t)));
        CR_CUDA(dt8.alloc(tris8.size() * sizeof(float)));
        CR_CUDA(cudaMemcpy(dn8.p, b8.nodes.data(), dn8.bytes, cudaMemcpyHostToDevice));
        CR_CUDA(cudaMemcpy(dt8.p, tris8.data(), dt8.bytes, cudaMemcpyHostToDevice));
    }
    DevMem dn4;
    if (bvh_flags & CR_BVH4) {
        CR_CUDA(dn4.alloc(b4.nodes.size() * sizeof(float)));
        CR_CUDA(cudaMemcpy(dn4.p, b4.nodes.data(), dn4.bytes, cudaMemcpyHostToDevice));
    }
    DevMem dl;
    const uint32_t n_lights = (uint32_t)lcdf.size();
    if (n_lights) {
        CR_CUDA(dl.alloc(lrec.size() * 4 + lcdf.size() * 4));
        CR_CUDA(cudaMemcpy(dl.p, lrec.data(), lrec.size() * 4, cudaMemcpyHostToDevice));
        CR_CUDA(cudaMemcpy(static_cast<char*>(dl.p) + lrec.size() * 4, lcdf.data(), lcdf.size() * 4,
                           cudaMemcpyHostToDevice));
    }
    s->d_lights = dl.p;
    dl.p = nullptr;
    s->dev.lights = static_cast<const float4*>(s->d_lights);
    s->dev.light_cdf = n_lights ? reinterpret_cast<const float*>(static_cast<const char*>(s->d_lights) + lrec.size() * 4)
                                : nullptr;
    s->dev.n_lights = n_lights;
    s->dev.light_total = n_lights ? lcdf.back() : 0.0f;
    s->d_nodes2 = dn.p;
    s->d_tris = dt.p;
    s->d_mats = dm.p;
    s->d_nodes8 = dn8.p;
    s->d_tris8 = dt8.p;
    s->d_nodes4 = dn4.p;
    dn.p = dt.p = dm.p = dn8.p = dt8.p = dn4.p = nullptr;
    s->dev.nodes4 = static_cast<const float4*>(s->d_nodes4);
    s->dev.n_nodes4 = b4.n_nodes;
    s->dev.nodes8 = static_cast<const uint4*>(s->d_nodes8);
    s->dev.tris8 = static_cast<const float4*>(s->d_tris8);
    s->dev.nodes2 = static_cast<const float4*>(s->d_nodes2);
    s->dev.tris = static_cast<const float4*>(s->d_tris);
    s->dev.mats = static_cast<const float4*>(s->d_mats);
    for (int k = 0; k < 3; ++k) {
        s->dev.env[k] = env ? env->radiance[k] : 0.0f;
        s->dev.lo[k] = b2.lo[k];
        s->dev.hi[k] = b2.hi[k];
    }
    s->dev.n_tri = n_tri;
    s->dev.n_mat = n_mat;
    s->dev.n_nodes2 = b2.n_nodes;
    s->dev.n_nodes8 = (bvh_flags & CR_BVH8Q) ? b8.n_nodes : 0u;
    {
        // the two scene-table entries, then the scene's error word (index checks of a debug build)
        DevMem de;
        CR_CUDA(de.alloc(2 * sizeof(SceneDev) + 16));
        s->dev.err = reinterpret_cast<uint32_t*>(static_cast<char*>(de.p) + 2 * sizeof(SceneDev));
        CR_CUDA(cudaMemset(s->dev.err, 0, 4));
        SceneDev ent[2] = {scene_entry(s->dev, false), scene_entry(s->dev, s->dev.nodes8 != nullptr)};
        ent[0].n_nodes4 = ent[1].n_nodes4 = s->dev.n_nodes4;
        CR_CUDA(cudaMemcpy(de.p, ent, sizeof(ent), cudaMemcpyHostToDevice));
        s->d_entries = static_cast<SceneDev*>(de.p);
        de.p = nullptr;
    }
    std::memset(&s->info, 0, sizeof(s->info));
    s->info.n_tri = n_tri;
    s->info.n_mat = n_mat;
    s->info.n_nodes2 = b2.n_nodes;
    s->info.depth2 = b2.depth;
    s->info.n_nodes8 = b8.n_nodes;
    s->info.n_nodes4 = b4.n_nodes;
    s->info.depth4 = b4.depth;
    s->info.device_bytes = b2.nodes.size() * 4 + tris.size() * 4 + mt.size() * 4 + b8.nodes.size() * 4 + tris8.size() * 4 +
                           b4.nodes.size() * 4 + lrec.size() * 4 + lcdf.size() * 4;
    s->info.n_lights = n_lights;
    s->info.light_area = s->dev.light_total;
    s->info.build_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    for (int k = 0; k < 3; ++k) {
        s->info.bounds_lo[k] = b2.lo[k];
        s->info.bounds_hi[k] = b2.hi[k];
    }
    *out = s.release();
    return CR_OK;
}

static void free_workspace(cr_scene* s) {
    s->ws.release();
    s->plan_dev.release();
    if (s->d_out) cudaFree(s->d_out);
    s->d_out = nullptr;
    s->out_cap = 0;
}

extern "C" cr_status cr_scene_destroy(cr_scene* s) {
    g_err.clear();
    if (!s) return CR_OK;
    cudaDeviceSynchronize();
    free_workspace(s);
    if (s->d_nodes2) cudaFree(s->d_nodes2);
    if (s->d_nodes8) cudaFree(s->d_nodes8);
    if (s->d_nodes4) cudaFree(s->d_nodes4);
    if (s->d_tris) cudaFree(s->d_tris);
    if (s->d_tris8) cudaFree(s->d_tris8);
    if (s->d_mats) cudaFree(s->d_mats);
    if (s->d_lights) cudaFree(s->d_lights);
    if (s->d_entries) cudaFree(s->d_entries);
    delete s;
    return CR_OK;
}

extern "C" cr_status cr_scene_get_info(const cr_scene* s, cr_scene_info* info) {
    g_err.clear();
    if (!s || !info) return fail(CR_ERR_INVALID_ARG, "cr_scene_get_info: NULL argument");
    *info = s->info;
    return CR_OK;
}

extern "C" cr_status cr_render_opts_default(cr_render_opts* o) {
    g_err.clear();
    if (!o) return fail(CR_ERR_INVALID_ARG, "cr_render_opts_default: NULL");
    std::memset(o, 0, sizeof(*o));
    o->interleave = 1;
    o->bvh = CR_BVH2;
    return CR_OK;
}

static bool pow2(uint32_t x) { return x && !(x & (x - 1)); }

static cr_status check_camera(const cr_camera* cam) {
    if (!cam) return fail(CR_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width == 0 || cam->height == 0 || (uint64_t)cam->width * cam->height > (1ull << 26))
        return fail(CR_ERR_INVALID_ARG, "camera size %ux%u out of range", cam->width, cam->height);
    if (!(cam->vfov_deg > 0.0f && cam->vfov_deg < 180.0f))
        return fail(CR_ERR_INVALID_ARG, "camera vfov %g not in (0, 180)", cam->vfov_deg);
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(cam->pos[k]) || !std::isfinite(cam->look_at[k]) || !std::isfinite(cam->up[k]))
            return fail(CR_ERR_INVALID_ARG, "camera has a non-finite coordinate");
    const float f[3] = {cam->look_at[0] - cam->pos[0], cam->look_at[1] - cam->pos[1], cam->look_at[2] - cam->pos[2]};
    const float c[3] = {f[1] * cam->up[2] - f[2] * cam->up[1], f[2] * cam->up[0] - f[0] * cam->up[2],
                        f[0] * cam->up[1] - f[1] * cam->up[0]};
    if (c[0] == 0.0f && c[1] == 0.0f && c[2] == 0.0f)
        return fail(CR_ERR_INVALID_ARG, "camera up is parallel to the view direction (or look_at == pos)");
    return CR_OK;
}

// Per-stage CUDA events recorded on the render stream without host synchronisation; the
// elapsed times are read once, after the stream has finished.
struct StageEvents {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<size_t, double*>> marks; // (index of start event, accumulator)
    cudaEvent_t get() {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pool.push_back(e);
        return e;
    }
    bool traces_only = false; // record only the trace stages (fewer event records in the step)
    // Every stage is also an NVTX range named after it (host enqueue time; a no-op unless a
    // tool is attached), so profilers can filter by stage.
    void begin(cudaStream_t s, double* acc, const char* name, bool is_trace = false) {
        nvtxRangePushA(name);
        if (!on || (traces_only && !is_trace)) return;
        st = s;
        cudaEvent_t e = get();
        if (!e) return;
        cudaEventRecord(e, st);
        marks.emplace_back(pool.size() - 1, acc);
    }
    void end() {
        nvtxRangePop();
        if (!on || marks.empty() || marks.back().first != pool.size() - 1) return;
        cudaEvent_t e = get();
        if (e) cudaEventRecord(e, st);
    }
    void resolve() {
        for (auto& m : marks) {
            if (m.first + 1 >= pool.size()) continue;
            float ms = 0;
            if (cudaEventElapsedTime(&ms, pool[m.first], pool[m.first + 1]) == cudaSuccess) *m.second += ms;
        }
    }
    ~StageEvents() {
        for (auto e : pool) cudaEventDestroy(e);
    }
};

namespace cr {

void Workspace::release() {
    if (base) cudaFree(base);
    base = nullptr;
    bytes = 0;
    pb = PathBuffers();
    if (phase_base) cudaFree(phase_base);
    phase_base = nullptr;
    phase_slots = 0;
    phase = PhaseBuffers();
    if (nee_base) cudaFree(nee_base);
    nee_base = nullptr;
    nee_slots = 0;
}

// Shadow-ray records of next-event estimation (48 bytes per slot), allocated after ensure().
cr_status Workspace::ensure_nee(uint32_t n_slots) {
    if (nee_base && nee_slots >= n_slots && pb.shadow_d) return CR_OK;
    if (nee_base) cudaFree(nee_base);
    nee_base = nullptr;
    nee_slots = 0;
    cudaError_t e = cudaMalloc(&nee_base, 48 * (size_t)n_slots);
    if (e != cudaSuccess) {
        cudaGetLastError();
        nee_base = nullptr;
        pb.shadow_o = pb.shadow_d = pb.shadow_c = nullptr;
        return fail(CR_ERR_OOM, "shadow-ray buffers: %s", cudaGetErrorString(e));
    }
    float4* f = static_cast<float4*>(nee_base);
    pb.shadow_o = f;
    pb.shadow_d = f + n_slots;
    pb.shadow_c = f + 2 * (size_t)n_slots;
    nee_slots = n_slots;
    return CR_OK;
}

#ifndef CR_PHASE_BUDGET
#define CR_PHASE_BUDGET 32 // node and leaf visits of the two-phase trace's first phase
#endif

cr_status Workspace::ensure_phase(uint32_t n_slots) {
    if (phase_base && phase_slots >= n_slots) return CR_OK;
    if (phase_base) cudaFree(phase_base);
    phase_base = nullptr;
    const size_t ns = n_slots, nb = (ns + 255) / 256 + 1;
    const size_t o_state = 0, o_susp = o_state + sizeof(TraceState) * ns, o_q2 = (o_susp + ns + 255) & ~(size_t)255,
                 o_cnt = (o_q2 + 4 * ns + 255) & ~(size_t)255, o_bc = o_cnt + 256, total = o_bc + 8 * nb;
    cudaError_t e = cudaMalloc(&phase_base, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        phase_base = nullptr;
        return fail(CR_ERR_OOM, "two-phase trace buffers: %s", cudaGetErrorString(e));
    }
    char* c = static_cast<char*>(phase_base);
    phase.state = reinterpret_cast<TraceState*>(c + o_state);
    phase.susp = reinterpret_cast<uint8_t*>(c + o_susp);
    phase.queue2 = reinterpret_cast<int32_t*>(c + o_q2);
    phase.count2 = reinterpret_cast<uint32_t*>(c + o_cnt);
    phase.block_counts = reinterpret_cast<uint32_t*>(c + o_bc);
    phase_slots = n_slots;
    return CR_OK;
}

// Carve the path state for n_slots slots and npx accumulation pixels out of one allocation.
cr_status Workspace::ensure(uint32_t n_slots, uint32_t npx) {
    if (base && pb.n_slots >= n_slots && pb.n_px_cap >= npx) return CR_OK;
    cudaDeviceSynchronize();
    release();
    const size_t ns = n_slots, np = npx;
    const size_t n_cblocks = compact_blocks(n_slots) + 1;
    const size_t n_hist = sort_hist_len(n_slots);
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += (b + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_pixel = take(4 * ns), o_job = take(2 * ns), o_scene = take(2 * ns), o_ro = take(16 * ns),
                 o_rd = take(16 * ns), o_hit = take(8 * ns), o_beta = take(16 * ns), o_rad = take(16 * ns),
                 o_alive = take(ns), o_rq = take(4 * ns), o_gq = take(2 * 4 * ns), o_counts = take(4 * kCountsWords),
                 o_bc = take(2 * 4 * n_cblocks), o_keys = take(2 * 4 * ns), o_vals = take(2 * 4 * ns),
                 o_hist = take(4 * n_hist), o_acc = take(16 * np);
    cudaError_t e = cudaMalloc(&base, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        base = nullptr;
        return fail(CR_ERR_OOM, "render workspace of %zu bytes: %s", off, cudaGetErrorString(e));
    }
    char* c = static_cast<char*>(base);
    bytes = off;
    pb.n_slots = n_slots;
    pb.n_px_cap = npx;
    pb.pixel = reinterpret_cast<int32_t*>(c + o_pixel);
    pb.slot_job = reinterpret_cast<uint16_t*>(c + o_job);
    pb.slot_scene = reinterpret_cast<uint16_t*>(c + o_scene);
    pb.ray_o = reinterpret_cast<float4*>(c + o_ro);
    pb.ray_d = reinterpret_cast<float4*>(c + o_rd);
    pb.hit = reinterpret_cast<int2*>(c + o_hit);
    pb.beta = reinterpret_cast<float4*>(c + o_beta);
    pb.radiance = reinterpret_cast<float4*>(c + o_rad);
    pb.alive = reinterpret_cast<uint8_t*>(c + o_alive);
    pb.ray_queue = reinterpret_cast<int32_t*>(c + o_rq);
    pb.group_queue = reinterpret_cast<int32_t*>(c + o_gq);
    pb.counts = reinterpret_cast<uint32_t*>(c + o_counts);
    pb.block_counts = reinterpret_cast<uint32_t*>(c + o_bc);
    pb.n_blocks_cap = (uint32_t)n_cblocks;
    pb.keys = reinterpret_cast<uint32_t*>(c + o_keys);
    pb.vals = reinterpret_cast<int32_t*>(c + o_vals);
    pb.sort_hist = reinterpret_cast<uint32_t*>(c + o_hist);
    pb.sort_hist_cap = (uint32_t)n_hist;
    pb.accum = reinterpret_cast<float4*>(c + o_acc);
    pb.counters = reinterpret_cast<unsigned long long*>(pb.counts + kCounterWord);
    return CR_OK;
}

cr_status queue_status(const uint64_t* host_counts) {
    const uint32_t e = reinterpret_cast<const uint32_t*>(host_counts)[kQueueErrWord];
    if (e & 1u) return fail(CR_ERR_CUDA, "queue compaction: an append would overflow a queue");
    if (e & 2u) return fail(CR_ERR_TIMEOUT, "ray sort: a grid-barrier wait ran out (the sorted order may be wrong)");
    return CR_OK;
}

// Device bytes of path state for n_slots slots and npx pixels (what Workspace::ensure takes).
size_t workspace_bytes(uint32_t n_slots, uint32_t npx) {
    const size_t ns = n_slots;
    return ns * (4 + 2 + 2 + 16 + 16 + 8 + 16 + 16 + 1 + 4 + 8 + 8 + 8) + 16ull * npx +
           4ull * sort_hist_len(n_slots) + 8ull * (compact_blocks(n_slots) + 1) + 4 * kCountsWords + 17 * 256;
}

// Check one job and fill the part of its device entry that does not depend on the pass.
cr_status check_job(const cr_job& j, uint32_t tile_w, uint32_t tile_h) {
    if (!j.scene) return fail(CR_ERR_INVALID_ARG, "job scene is NULL");
    cr_status st = check_camera(&j.camera);
    if (st != CR_OK) return st;
    if (j.spp == 0) return fail(CR_ERR_INVALID_ARG, "spp must be >= 1");
    if (j.max_bounces == 0 || j.max_bounces > 16)
        return fail(CR_ERR_INVALID_ARG, "max_bounces %u not in [1, 16]", j.max_bounces);
    if (j.mode > CR_WORLD_REUSE) return fail(CR_ERR_INVALID_ARG, "unknown mode %u", j.mode);
    if (j.flags & ~(uint32_t)(CR_JOB_NEE | CR_JOB_HYBRID_DONOR | CR_JOB_NEE_SHARED))
        return fail(CR_ERR_INVALID_ARG, "unknown job flags 0x%x", j.flags);
    if (!(j.diffuse_roughness >= 0.0f) || !std::isfinite(j.diffuse_roughness))
        return fail(CR_ERR_INVALID_ARG, "diffuse_roughness %g not finite and >= 0", (double)j.diffuse_roughness);
    (void)tile_w;
    (void)tile_h;
    return CR_OK;
}

// Build the per-pass job tables of a set of jobs that share the tile shape and K.
// The device entry of sample `sample` of a job (tile_base, slot_tile and px_base are the
// caller's: they place the job in a pass and its buffers).
JobDev job_dev(const cr_job& j, const PlanOpts& po, uint32_t scene_idx, uint32_t sample) {
    JobDev d;
    std::memset(&d, 0, sizeof(d));
    d.cam = make_camera(j.camera);
    d.tiles_x = (j.camera.width + po.tile_w - 1) / po.tile_w;
    d.scene = scene_idx;
    d.frame = j.frame_base + sample;
    d.max_bounces = j.max_bounces;
    d.reuse_mask = 0;
    d.world_mask = 0;
    for (uint32_t b = 1; b <= j.max_bounces; ++b)
        if (j.reuse_depth == 0 || b <= j.reuse_depth) {
            if (j.mode == CR_DIRECTION_REUSE) d.reuse_mask |= 1u << b;
            if (j.mode == CR_WORLD_REUSE) d.world_mask |= 1u << b;
        }
    d.interleave = po.interleave ? 1u : 0u;
    d.nee = (j.flags & CR_JOB_NEE) ? ((j.flags & CR_JOB_NEE_SHARED) ? 2u : 1u) : 0u;
    d.hybrid_donor = (j.flags & CR_JOB_HYBRID_DONOR) ? 1u : 0u;
    d.seed = j.seed;
    d.out = j.out_rgb;
    d.inv_spp = 1.0f / (float)j.spp;
    d.sample_flags = (sample == 0 ? 1u : 0u) | (sample + 1 == j.spp ? 2u : 0u);
    d.diffuse_rough = j.diffuse_roughness;
    return d;
}

cr_status build_plan(const cr_job* jobs, uint32_t n_jobs, const PlanOpts& po, RenderPlan& plan) {
    if (n_jobs == 0 || n_jobs > 65535) return fail(CR_ERR_INVALID_ARG, "n_jobs %u not in [1, 65535]", n_jobs);
    const uint32_t m = po.tile_w * po.tile_h;
    if (po.tile_w == 0 || po.tile_h == 0 || !pow2(m) || m > 1024)
        return fail(CR_ERR_INVALID_ARG, "group_w*group_h = %ux%u must be a power of two <= 1024", po.tile_w, po.tile_h);
    const uint32_t K = po.k ? po.k : m;
    if (!pow2(K) || m % K != 0 || K > 256)
        return fail(CR_ERR_INVALID_ARG, "K=%u must be a power of two dividing W*H=%u and <= 256", K, m);
    plan = RenderPlan();
    plan.tile_w = po.tile_w;
    plan.tile_h = po.tile_h;
    plan.m = m;
    plan.k = K;
    plan.bvh8 = po.bvh8;
    plan.bvh4 = po.bvh4;
    // scene table
    std::vector<const cr_scene*> uniq;
    std::vector<uint32_t> scene_idx(n_jobs);
    uint32_t max_spp = 0, px = 0;
    for (uint32_t i = 0; i < n_jobs; ++i) {
        cr_status st = check_job(jobs[i], po.tile_w, po.tile_h);
        if (st != CR_OK) return st;
        if (po.bvh8 && !jobs[i].scene->dev.nodes8)
            return fail(CR_ERR_INVALID_ARG, "job %u: the scene has no BVH8-Q (create it with CR_BVH8Q)", i);
        if (po.bvh4 && !jobs[i].scene->dev.nodes4)
            return fail(CR_ERR_INVALID_ARG, "job %u: the scene has no BVH4 (create it with CR_BVH4)", i);
        uint32_t k = 0;
        while (k < uniq.size() && uniq[k] != jobs[i].scene) ++k;
        if (k == uniq.size()) uniq.push_back(jobs[i].scene);
        scene_idx[i] = k;
        max_spp = std::max(max_spp, jobs[i].spp);
        plan.max_bounces = std::max(plan.max_bounces, jobs[i].max_bounces);
        if (jobs[i].mode == CR_MORTON_SORT) plan.sort = true;
        px += jobs[i].camera.width * jobs[i].camera.height;
        if ((uint64_t)px > (1ull << 28)) return fail(CR_ERR_INVALID_ARG, "too many pixels in the batch");
    }
    for (auto* sc : uniq) {
        plan.scenes.push_back(scene_entry(sc->dev, po.bvh8));
        plan.scenes.back().n_nodes4 = sc->dev.n_nodes4;
    }
    plan.npx_total = px;
    // passes: pass p renders sample p of every job with spp > p
    uint32_t px_base = 0;
    std::vector<uint32_t> pxb(n_jobs);
    for (uint32_t i = 0; i < n_jobs; ++i) {
        pxb[i] = px_base;
        px_base += jobs[i].camera.width * jobs[i].camera.height;
    }
    if (po.tile_end != 0) {
        const cr_job& j = jobs[0];
        const uint64_t all = (uint64_t)((j.camera.width + po.tile_w - 1) / po.tile_w) *
                             ((j.camera.height + po.tile_h - 1) / po.tile_h);
        if (n_jobs != 1 || po.tile_begin >= po.tile_end || po.tile_end > all)
            return fail(CR_ERR_INVALID_ARG, "tile range [%u, %u) is not within the image's %llu tiles", po.tile_begin,
                        po.tile_end, (unsigned long long)all);
    }
    for (uint32_t p = 0; p < max_spp; ++p) {
        Pass ps;
        ps.job_offset = (uint32_t)plan.jobs.size();
        uint32_t tiles = 0;
        for (uint32_t i = 0; i < n_jobs; ++i) {
            const cr_job& j = jobs[i];
            if (j.spp <= p) continue;
            JobDev d = job_dev(j, po, scene_idx[i], p);
            const uint32_t tiles_y = (j.camera.height + po.tile_h - 1) / po.tile_h;
            d.tile_base = tiles;
            d.slot_tile = tiles;
            d.px_base = pxb[i];
            if (d.nee) plan.nee = true;
            uint64_t job_tiles = (uint64_t)d.tiles_x * tiles_y;
            if (po.tile_end != 0) {
                d.tile_first = po.tile_begin;
                job_tiles = po.tile_end - po.tile_begin;
            }
            const uint64_t t64 = (uint64_t)tiles + job_tiles;
            if (t64 * m > (1ull << 27)) return fail(CR_ERR_INVALID_ARG, "pass %u: too many slots", p);
            tiles = (uint32_t)t64;
            plan.jobs.push_back(d);
        }
        ps.n_jobs = (uint32_t)plan.jobs.size() - ps.job_offset;
        ps.n_tiles = tiles;
        plan.max_slots = std::max(plan.max_slots, tiles * m);
        plan.passes.push_back(ps);
    }
    return CR_OK;
}

cr_status Plan::upload(const RenderPlan& p, cudaStream_t st) {
    size_t bj = sizeof(JobDev) * p.jobs.size(), bs = sizeof(SceneDev) * p.scenes.size();
    cudaError_t e = cudaSuccess;
    if (bj > cap_jobs || bs > cap_scenes) { // grow (the tables are reused across calls)
        cudaDeviceSynchronize();
        release();
        e = cudaMalloc(&d_jobs, bj);
        if (e == cudaSuccess) e = cudaMalloc(&d_scenes, bs);
        if (e != cudaSuccess) {
            cudaGetLastError();
            release();
            return fail(CR_ERR_OOM, "job tables: %s", cudaGetErrorString(e));
        }
        cap_jobs = bj;
        cap_scenes = bs;
    }
    e = cudaMemcpyAsync(d_jobs, p.jobs.data(), bj, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_scenes, p.scenes.data(), bs, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(CR_ERR_CUDA, "job tables: %s", cudaGetErrorString(e));
    return CR_OK;
}

void Plan::release() {
    if (d_jobs) cudaFree(d_jobs);
    if (d_scenes) cudaFree(d_scenes);
    d_jobs = nullptr;
    d_scenes = nullptr;
    cap_jobs = cap_scenes = 0;
}

// Enqueue every stage of a plan on one stream (all passes, all bounces, then the output).
// Nothing here synchronises the host, so the sequence can also be captured into a graph.
cr_status enqueue_plan(const RenderPlan& p, const Plan& dev, Workspace& ws, const ExecOpts& eo, cudaStream_t stream,
                       LaunchCount& lc, StageTimes* times) {
    PathBuffers& b = ws.pb;
    StageEvents ev;
    ev.on = times != nullptr;
    ev.traces_only = eo.stats_traces_only;
    cr_status failst = CR_OK;
    auto check = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && failst == CR_OK) failst = fail(CR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    };
    check(cudaMemsetAsync(b.counts, 0, 4 * kCountsWords, stream), "memset counts");
    // a fresh render writes its first samples' sums and its outputs from the accumulation
    // kernel; otherwise (the server's resident sums) the buffer is cleared / output as asked
    const bool fused_out = eo.clear_accum && eo.write_output;
    if (eo.clear_accum && !fused_out)
        check(cudaMemsetAsync(b.accum, 0, 16 * (size_t)p.npx_total, stream), "memset accum");
    TraceArgs ta;
    ta.ray_o = b.ray_o;
    ta.ray_d = b.ray_d;
    ta.hit = b.hit;
    ta.block = eo.block;
    ta.stack = eo.stack;
    ta.persistent = eo.persistent;
    ta.speculative = eo.speculative;
    ta.work_counter = b.counts + 2;
    ta.bvh8 = p.bvh8;
    ta.bvh4 = p.bvh4;
    ta.scenes = dev.d_scenes;
    ta.slot_scene = b.slot_scene;
    double dummy = 0.0;
    for (const Pass& ps : p.passes) {
        PassArgs P;
        P.jobs = dev.d_jobs + ps.job_offset;
        P.n_jobs = ps.n_jobs;
        P.scenes = dev.d_scenes;
        P.tile_w = p.tile_w;
        P.tile_h = p.tile_h;
        P.m = p.m;
        P.k = p.k;
        P.n_tiles = ps.n_tiles;
        P.npx = eo.debug_npx;
        P.nee = p.nee;
        P.accum_mode = fused_out ? 3u : 0u;
        const uint32_t n_slots = ps.n_tiles * p.m;
        b.n_groups = n_slots / p.k;
        ev.begin(stream, times ? &times->raygen : &dummy, "cr raygen");
        launch_raygen(P, b, stream, lc);
        ev.end();
        ta.queue = primary_pixel_order() ? b.ray_queue : nullptr; // written by raygen: pixel order per tile
        ta.queue_count = nullptr;
        ta.n_max = n_slots;
        ta.counters = nullptr;
        if (ta.persistent) check(cudaMemsetAsync(ta.work_counter, 0, 4, stream), "memset");
        ta.packet = eo.packet_primary;
        ta.block = eo.block;
        ev.begin(stream, times ? &times->trace_primary : &dummy, "cr trace primary", true);
        launch_trace(ta, stream, lc);
        ev.end();
        ta.packet = eo.packet_secondary;
        ta.block = eo.block_secondary ? eo.block_secondary : eo.block;
        for (uint32_t bnc = 1; bnc <= p.max_bounces; ++bnc) {
            P.bounce = bnc;
            ev.begin(stream, times ? &times->shade : &dummy, "cr shade");
            launch_shade(P, b, bnc == 1, !eo.ordered_queues, eo.debug, stream, lc);
            ev.end();
            if (P.nee && b.shadow_d) {
                ev.begin(stream, times ? &times->trace_shadow : &dummy, "cr trace shadow", true);
                launch_shadow(P, b, bnc == 1, p.bvh8, stream, lc);
                ev.end();
            }
            if (eo.ordered_queues) {
                ev.begin(stream, times ? &times->compact : &dummy, "cr compact");
                launch_compact(P, b, bnc == 1, stream, lc);
                ev.end();
            }
            ta.queue = b.ray_queue;
            ta.queue_count = b.counts + 8 + 2 * bnc;
            ta.n_max = n_slots;
            if (p.sort) {
                ev.begin(stream, times ? &times->sort : &dummy, "cr sort");
                ta.queue = launch_morton_sort(P, b, bnc, eo.sort_key, stream, lc);
                ev.end();
            }
            ta.counters = eo.count ? b.counters : nullptr;
            if (ta.persistent) check(cudaMemsetAsync(ta.work_counter, 0, 4, stream), "memset");
            ta.two_phase = eo.phase_budget > 0 && ws.phase.state;
            ta.phase = ws.phase;
            ta.phase.budget = eo.phase_budget;
            ev.begin(stream, times ? &times->trace_secondary : &dummy, "cr trace secondary", true);
            launch_trace(ta, stream, lc);
            ev.end();
        }
        P.bounce = p.max_bounces + 1;
        ev.begin(stream, times ? &times->accum : &dummy, "cr accumulate");
        launch_finish_accumulate(P, b, eo.debug, stream, lc);
        ev.end();
    }
    // pass 0 holds every job (spp >= 1), with the px_base and output of each
    if (eo.write_output && !fused_out)
        launch_output(dev.d_jobs, p.passes[0].n_jobs, b.accum, p.npx_total, stream, lc);
    check(cudaGetLastError(), "launch");
    if (times) {
        // the caller synchronises the stream before reading; resolve needs completed events
        check(cudaStreamSynchronize(stream), "sync");
        ev.resolve();
    }
    return failst;
}

} // namespace cr

extern "C" cr_status cr_render_ex(cr_scene* s, const cr_camera* cam, uint32_t spp, uint32_t max_bounces,
                                  cr_reuse_mode mode, uint32_t group_w, uint32_t group_h, float* out_rgb,
                                  const cr_render_opts* opts_in) {
    g_err.clear();
    if (!s) return fail(CR_ERR_INVALID_ARG, "cr_render: scene is NULL");
    if (!out_rgb) return fail(CR_ERR_INVALID_ARG, "cr_render: out_rgb is NULL");
    cr_render_opts o;
    cr_render_opts_default(&o);
    if (opts_in) o = *opts_in;
    const bool use8 = o.bvh == CR_BVH8Q, use4 = o.bvh == CR_BVH4;
    if ((o.bvh != CR_BVH2 && o.bvh != 0 && !use8 && !use4) || (use8 && !s->dev.nodes8) || (use4 && !s->dev.nodes4))
        return fail(CR_ERR_INVALID_ARG, "cr_render: bvh %u not available for this scene", o.bvh);
    const int block = o.block ? (int)o.block : 128;
    if (block % 32 != 0 || block < 32 || block > 512) return fail(CR_ERR_INVALID_ARG, "cr_render: block %d", block);
    if (o.debug && spp != 1) return fail(CR_ERR_INVALID_ARG, "cr_render: debug capture needs spp == 1");
    if (o.debug && (!o.debug->prim || !o.debug->cat || !o.debug->cls || !o.debug->flags || !o.debug->local || !o.debug->world))
        return fail(CR_ERR_INVALID_ARG, "cr_render: debug capture needs all six buffers");
    if (o.debug && (!o.debug->ray != !o.debug->t || !o.debug->ray != !o.debug->beta))
        return fail(CR_ERR_INVALID_ARG, "cr_render: replay capture needs ray, t and beta together");
    cudaStream_t stream = static_cast<cudaStream_t>(o.stream);
    cr_status st = check_camera(cam);
    if (st != CR_OK) return st;
    const bool out_dev = is_device_ptr(out_rgb);
    if (!out_dev && (o.flags & CR_OPT_NO_SYNC))
        return fail(CR_ERR_INVALID_ARG, "cr_render: CR_OPT_NO_SYNC needs a device out_rgb");
    const uint32_t npx = cam->width * cam->height;
    if (!out_dev && s->out_cap < (size_t)npx * 3) {
        if (s->d_out) cudaFree(s->d_out);
        s->d_out = nullptr;
        s->out_cap = 0;
        CR_CUDA(cudaMalloc(&s->d_out, sizeof(float) * 3 * (size_t)npx));
        s->out_cap = (size_t)npx * 3;
    }
    cr_job job;
    std::memset(&job, 0, sizeof(job));
    job.scene = s;
    job.camera = *cam;
    job.spp = spp;
    job.max_bounces = max_bounces;
    job.mode = (uint32_t)mode;
    job.reuse_depth = o.reuse_depth;
    job.seed = o.seed;
    job.frame_base = o.frame_base;
    job.diffuse_roughness = o.diffuse_roughness;
    job.flags = ((o.flags & CR_OPT_NEE) ? (uint32_t)CR_JOB_NEE : 0u) |
                ((o.flags & CR_OPT_HYBRID_DONOR) ? (uint32_t)CR_JOB_HYBRID_DONOR : 0u) |
                ((o.flags & CR_OPT_NEE_SHARED) ? (uint32_t)CR_JOB_NEE_SHARED : 0u);
    job.out_rgb = out_dev ? out_rgb : s->d_out;
    PlanOpts po;
    po.tile_w = group_w;
    po.tile_h = group_h;
    po.k = o.k;
    po.interleave = o.interleave;
    po.bvh8 = use8;
    po.bvh4 = use4;
    if (o.tile_begin != 0 || o.tile_end != 0) {
        po.tile_begin = o.tile_begin;
        po.tile_end = o.tile_end;
        if (po.tile_end == 0) return fail(CR_ERR_INVALID_ARG, "cr_render: tile_end is 0 with tile_begin %u", o.tile_begin);
    }
    RenderPlan plan;
    st = build_plan(&job, 1, po, plan);
    if (st != CR_OK) return st;
    st = s->ws.ensure(plan.max_slots, plan.npx_total);
    if (st != CR_OK) return st;
    if (plan.nee) {
        st = s->ws.ensure_nee(plan.max_slots);
        if (st != CR_OK) return st;
    }
    Plan& dev = s->plan_dev;
    st = dev.upload(plan, stream);
    if (st != CR_OK) return st;
    ExecOpts eo;
    eo.block = block;
    eo.block_secondary = o.block ? block : kSecondaryBlock;
    if (o.stack != 0 && o.stack != 8 && o.stack != 16 && o.stack != 32)
        return fail(CR_ERR_INVALID_ARG, "cr_render: stack %u not in {8, 16, 32}", o.stack);
    eo.stack = o.stack ? o.stack : 16;
    eo.persistent = (o.flags & CR_OPT_PERSISTENT) != 0;
    eo.speculative = (o.flags & CR_OPT_SPECULATIVE) != 0;
    eo.packet_primary = (o.flags & CR_OPT_PACKET_PRIMARY) != 0;
    eo.packet_secondary = (o.flags & CR_OPT_PACKET_SECONDARY) != 0;
    eo.count = (o.flags & CR_OPT_COUNT) != 0;
    if (o.sort_key > CR_SORT_HIERARCHY_CUT) return fail(CR_ERR_INVALID_ARG, "cr_render: sort_key %u", o.sort_key);
    eo.sort_key = o.sort_key;
    if (o.flags & CR_OPT_TWO_PHASE) {
        eo.phase_budget = CR_PHASE_BUDGET;
        st = s->ws.ensure_phase(plan.max_slots);
        if (st != CR_OK) return st;
    }
    eo.debug = o.debug;
    eo.debug_npx = npx;
    eo.stats_traces_only = (o.flags & CR_OPT_STATS_TRACES) && !(o.flags & CR_OPT_STATS);
    eo.ordered_queues = (o.flags & CR_OPT_ORDERED_QUEUES) != 0;
    LaunchCount lc;
    StageTimes times;
    cudaEvent_t e_all[2];
    if (o.stats) {
        CR_CUDA(cudaEventCreate(&e_all[0]));
        CR_CUDA(cudaEventCreate(&e_all[1]));
        CR_CUDA(cudaEventRecord(e_all[0], stream));
    }
    if (!out_dev && po.tile_end != 0) // pixels outside the range keep the caller's values
        CR_CUDA(cudaMemcpyAsync(s->d_out, out_rgb, sizeof(float) * 3 * (size_t)npx, cudaMemcpyHostToDevice, stream));
    st = enqueue_plan(plan, dev, s->ws, eo, stream, lc,
                      (o.stats && (o.flags & (CR_OPT_STATS | CR_OPT_STATS_TRACES))) ? &times : nullptr);
    if (st != CR_OK) return st;
    if (!out_dev) CR_CUDA(cudaMemcpyAsync(out_rgb, s->d_out, sizeof(float) * 3 * (size_t)npx, cudaMemcpyDeviceToHost, stream));
    if (o.stats) {
        cr_stats stats;
        std::memset(&stats, 0, sizeof(stats));
        CR_CUDA(cudaEventRecord(e_all[1], stream));
        uint64_t host_counts[kCountsWords / 2];
        CR_CUDA(cudaMemcpyAsync(host_counts, s->ws.pb.counts, 4 * kCountsWords, cudaMemcpyDeviceToHost, stream));
        CR_CUDA(cudaStreamSynchronize(stream));
        float ms = 0;
        cudaEventElapsedTime(&ms, e_all[0], e_all[1]);
        stats.ms_total = ms;
        stats.ms_raygen = times.raygen;
        stats.ms_trace_primary = times.trace_primary;
        stats.ms_trace_secondary = times.trace_secondary;
        stats.ms_shade = times.shade;
        stats.ms_compact = times.compact;
        stats.ms_sort = times.sort;
        stats.ms_accum = times.accum;
        const uint64_t* stat = host_counts + kStatWord / 2;
        for (uint32_t bb = 1; bb <= max_bounces; ++bb) stats.secondary_rays += stat[bb];
        stats.secondary_rays_b1 = stat[1];
        const uint64_t* ctr = host_counts + kCounterWord / 2;
        stats.node_visits = ctr[0];
        stats.tri_tests = ctr[1];
        stats.shadow_rays = host_counts[kShadowWord / 2];
        stats.ms_trace_shadow = times.trace_shadow;
        stats.h2d_bytes = sizeof(JobDev) * plan.jobs.size() + sizeof(SceneDev) * plan.scenes.size() +
                          ((!out_dev && po.tile_end != 0) ? sizeof(float) * 3 * (size_t)npx : 0);
        stats.d2h_bytes = out_dev ? 0 : sizeof(float) * 3 * (uint64_t)npx;
        stats.primary_rays = (uint64_t)npx * spp;
        stats.kernel_launches = lc.n;
        *o.stats = stats;
        cudaEventDestroy(e_all[0]);
        cudaEventDestroy(e_all[1]);
        st = queue_status(host_counts);
        if (st != CR_OK) return st;
    }
    if (!(o.flags & CR_OPT_NO_SYNC)) {
        CR_CUDA(cudaStreamSynchronize(stream));
        st = debug_word_status(s);
        if (st != CR_OK) return st;
    }
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

extern "C" cr_status cr_render(cr_scene* s, const cr_camera* cam, uint32_t spp, uint32_t max_bounces, cr_reuse_mode mode,
                               uint32_t group_w, uint32_t group_h, float* out_rgb) {
    return cr_render_ex(s, cam, spp, max_bounces, mode, group_w, group_h, out_rgb, nullptr);
}

// ------------------------------------------------------------------------------------
// Parity entry points.  Host arguments are staged through temporary device buffers.
namespace {
struct Staged {
    DevMem mem;
    void* dev = nullptr;
    bool host = false;
    void* user = nullptr;
    size_t bytes = 0;
};

cudaError_t stage_in(Staged& sb, const void* user, size_t bytes, cudaStream_t st) {
    sb.user = const_cast<void*>(user);
    sb.bytes = bytes;
    if (!user) return cudaSuccess;
    if (is_device_ptr(user)) {
        sb.dev = const_cast<void*>(user);
        return cudaSuccess;
    }
    sb.host = true;
    cudaError_t e = sb.mem.alloc(bytes);
    if (e != cudaSuccess) return e;
    sb.dev = sb.mem.p;
    return cudaMemcpyAsync(sb.dev, user, bytes, cudaMemcpyHostToDevice, st);
}
cudaError_t stage_out(Staged& sb, void* user, size_t bytes) {
    sb.user = user;
    sb.bytes = bytes;
    if (is_device_ptr(user)) {
        sb.dev = user;
        return cudaSuccess;
    }
    sb.host = true;
    cudaError_t e = sb.mem.alloc(bytes);
    sb.dev = sb.mem.p;
    return e;
}
cudaError_t finish_out(Staged& sb, cudaStream_t st) {
    if (!sb.host || !sb.user) return cudaSuccess;
    return cudaMemcpyAsync(sb.user, sb.dev, sb.bytes, cudaMemcpyDeviceToHost, st);
}
} // namespace

extern "C" cr_status cr_trace_rays(cr_scene* s, const float* rays, const int32_t* skip_prim, uint32_t n, int32_t* prim,
                                   float* t, const cr_render_opts* opts_in) {
    g_err.clear();
    if (!s || (!rays && n) || (!prim && n) || (!t && n)) return fail(CR_ERR_INVALID_ARG, "cr_trace_rays: NULL argument");
    if (n == 0) return CR_OK;
    if (n > (1u << 28)) return fail(CR_ERR_INVALID_ARG, "cr_trace_rays: n=%u too large", n);
    cr_render_opts o;
    cr_render_opts_default(&o);
    if (opts_in) o = *opts_in;
    const bool use8 = o.bvh == CR_BVH8Q, use4 = o.bvh == CR_BVH4;
    if ((o.bvh != CR_BVH2 && o.bvh != 0 && !use8 && !use4) || (use8 && !s->dev.nodes8) || (use4 && !s->dev.nodes4))
        return fail(CR_ERR_INVALID_ARG, "cr_trace_rays: bvh %u not available", o.bvh);
    const float4* tris = use8 ? s->dev.tris8 : s->dev.tris;
    const int block = o.block ? (int)o.block : 128;
    if (block % 32 != 0 || block < 32 || block > 512) return fail(CR_ERR_INVALID_ARG, "cr_trace_rays: block %d", block);
    cudaStream_t stream = static_cast<cudaStream_t>(o.stream);
    Staged r_in, s_in, p_out, t_out;
    CR_CUDA(stage_in(r_in, rays, sizeof(float) * 8 * (size_t)n, stream));
    CR_CUDA(stage_in(s_in, skip_prim, sizeof(int32_t) * (size_t)n, stream));
    CR_CUDA(stage_out(p_out, prim, sizeof(int32_t) * (size_t)n));
    CR_CUDA(stage_out(t_out, t, sizeof(float) * (size_t)n));
    DevMem ro, rd, hit, wc;
    CR_CUDA(ro.alloc(16 * (size_t)n));
    CR_CUDA(rd.alloc(16 * (size_t)n));
    CR_CUDA(hit.alloc(8 * (size_t)n));
    CR_CUDA(wc.alloc(16 * 4));
    CR_CUDA(cudaMemsetAsync(wc.p, 0, 64, stream));
    LaunchCount lc;
    launch_rays_from_user(r_in.dev ? static_cast<const float*>(r_in.dev) : nullptr,
                          static_cast<const int32_t*>(s_in.dev), n, ro.as<float4>(), rd.as<float4>(), stream, lc);
    TraceArgs ta;
    ta.ray_o = ro.as<float4>();
    ta.ray_d = rd.as<float4>();
    ta.hit = hit.as<int2>();
    ta.n_max = n;
    ta.block = block;
    ta.persistent = (o.flags & CR_OPT_PERSISTENT) != 0;
    ta.speculative = (o.flags & CR_OPT_SPECULATIVE) != 0;
    ta.packet = (o.flags & (CR_OPT_PACKET_PRIMARY | CR_OPT_PACKET_SECONDARY)) != 0;
    ta.any_hit = (o.flags & CR_OPT_ANY_HIT) != 0;
    ta.bvh8 = use8;
    ta.bvh4 = use4;
    ta.scenes = dev_scene_entry(s, use8);
    ta.slot_scene = nullptr;
    ta.work_counter = wc.as<uint32_t>();
    ta.counters = (o.flags & CR_OPT_COUNT) ? reinterpret_cast<unsigned long long*>(wc.as<uint32_t>() + 4) : nullptr;
    cudaEvent_t e0, e1;
    if (o.stats) {
        CR_CUDA(cudaEventCreate(&e0));
        CR_CUDA(cudaEventCreate(&e1));
        CR_CUDA(cudaEventRecord(e0, stream));
    }
    launch_trace(ta, stream, lc);
    if (o.stats) CR_CUDA(cudaEventRecord(e1, stream));
    launch_hits_to_user(tris, hit.as<int2>(), n, static_cast<int32_t*>(p_out.dev), static_cast<float*>(t_out.dev), stream, lc);
    CR_CUDA(cudaGetLastError());
    CR_CUDA(finish_out(p_out, stream));
    CR_CUDA(finish_out(t_out, stream));
    CR_CUDA(cudaStreamSynchronize(stream));
    {
        const cr_status dst = debug_word_status(s);
        if (dst != CR_OK) return dst;
    }
    if (o.stats) {
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        std::memset(o.stats, 0, sizeof(cr_stats));
        o.stats->ms_trace_secondary = ms;
        o.stats->ms_total = ms;
        o.stats->secondary_rays = n;
        o.stats->kernel_launches = lc.n;
        if (ta.counters) {
            unsigned long long c[2];
            CR_CUDA(cudaMemcpy(c, ta.counters, sizeof(c), cudaMemcpyDeviceToHost));
            o.stats->node_visits = c[0];
            o.stats->tri_tests = c[1];
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    return CR_OK;
}

extern "C" cr_status cr_debug_groups(uint32_t width, uint32_t height, uint32_t group_w, uint32_t group_h,
                                     uint32_t interleave, uint64_t seed, uint32_t frame, uint32_t* slot_of_pixel) {
    g_err.clear();
    const uint32_t m = group_w * group_h;
    if (!slot_of_pixel || !width || !height || (uint64_t)width * height > (1ull << 26))
        return fail(CR_ERR_INVALID_ARG, "cr_debug_groups: bad size or NULL output");
    if (!group_w || !group_h || !pow2(m) || m > 1024)
        return fail(CR_ERR_INVALID_ARG, "cr_debug_groups: W*H must be a power of two <= 1024");
    CamBasis cam;
    std::memset(&cam, 0, sizeof(cam));
    cam.width = width;
    cam.height = height;
    Staged out;
    const size_t bytes = sizeof(uint32_t) * (size_t)width * height;
    CR_CUDA(stage_out(out, slot_of_pixel, bytes));
    LaunchCount lc;
    launch_groups(cam, group_w, group_h, interleave ? 1u : 0u, seed, frame, static_cast<uint32_t*>(out.dev), 0, lc);
    CR_CUDA(cudaGetLastError());
    CR_CUDA(finish_out(out, 0));
    CR_CUDA(cudaStreamSynchronize(0));
    return CR_OK;
}

extern "C" cr_status cr_debug_philox(uint64_t seed, const uint32_t* ctr, uint32_t n, uint32_t* out) {
    g_err.clear();
    if (n == 0) return CR_OK;
    if (!ctr || !out) return fail(CR_ERR_INVALID_ARG, "cr_debug_philox: NULL argument");
    Staged ci, co;
    CR_CUDA(stage_in(ci, ctr, 16 * (size_t)n, 0));
    CR_CUDA(stage_out(co, out, 16 * (size_t)n));
    LaunchCount lc;
    launch_philox(seed, static_cast<const uint32_t*>(ci.dev), n, static_cast<uint32_t*>(co.dev), 0, lc);
    CR_CUDA(cudaGetLastError());
    CR_CUDA(finish_out(co, 0));
    CR_CUDA(cudaStreamSynchronize(0));
    return CR_OK;
}

extern "C" cr_status cr_debug_sort(const uint32_t* keys, const int32_t* vals, uint32_t n, uint32_t reps,
                                   uint32_t* keys_out, int32_t* vals_out, double* ms) {
    g_err.clear();
    if (n == 0) return CR_OK;
    if (!keys || !vals || !keys_out || !vals_out || reps == 0)
        return fail(CR_ERR_INVALID_ARG, "cr_debug_sort: NULL argument or reps == 0");
    if (n > (1u << 28)) return fail(CR_ERR_INVALID_ARG, "cr_debug_sort: n=%u above 2^28", n);
    Staged ki, vi, ko, vo;
    CR_CUDA(stage_in(ki, keys, 4 * (size_t)n, 0));
    CR_CUDA(stage_in(vi, vals, 4 * (size_t)n, 0));
    CR_CUDA(stage_out(ko, keys_out, 4 * (size_t)n));
    CR_CUDA(stage_out(vo, vals_out, 4 * (size_t)n));
    // the sort's own buffers: keys and values twice, the workspace, the count and error words
    DevMem buf;
    const size_t ws_words = sort_hist_len(n);
    CR_CUDA(buf.alloc(16 * (size_t)n + 4 * ws_words + 64));
    uint32_t* kk = static_cast<uint32_t*>(buf.p);
    int32_t* vv = reinterpret_cast<int32_t*>(kk + 2 * (size_t)n);
    uint32_t* ws = reinterpret_cast<uint32_t*>(vv + 2 * (size_t)n);
    uint32_t* cnt = ws + ws_words;
    const uint32_t host_cnt[2] = {n, 0u};
    CR_CUDA(cudaMemcpy(cnt, host_cnt, 8, cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CR_CUDA(cudaEventCreate(&e0));
    CR_CUDA(cudaEventCreate(&e1));
    LaunchCount lc;
    int32_t* sorted = nullptr;
    cudaEventRecord(e0, 0);
    for (uint32_t r = 0; r < reps; ++r)
        sorted = launch_sort_only(static_cast<const uint32_t*>(ki.dev), static_cast<const int32_t*>(vi.dev), n, kk, vv,
                                  ws, cnt, cnt + 1, 0, lc);
    cudaEventRecord(e1, 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float el = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&el, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CR_CUDA(e);
    if (ms) *ms = (double)el / reps;
    const uint32_t* sorted_keys = kk + (sorted - vv);
    CR_CUDA(cudaMemcpyAsync(ko.dev, sorted_keys, 4 * (size_t)n, cudaMemcpyDeviceToDevice, 0));
    CR_CUDA(cudaMemcpyAsync(vo.dev, sorted, 4 * (size_t)n, cudaMemcpyDeviceToDevice, 0));
    CR_CUDA(finish_out(ko, 0));
    CR_CUDA(finish_out(vo, 0));
    uint32_t err = 0;
    CR_CUDA(cudaMemcpy(&err, cnt + 1, 4, cudaMemcpyDeviceToHost));
    if (err) return fail(CR_ERR_TIMEOUT, "cr_debug_sort: a grid-barrier wait ran out");
    return CR_OK;
}

extern "C" cr_status cr_debug_sample(uint32_t kind, uint32_t n, const float* wo, const float* u, const float* param,
                                     float* wi, float* weight, uint8_t* valid) {
    g_err.clear();
    if (n == 0) return CR_OK;
    if (kind > 3) return fail(CR_ERR_INVALID_ARG, "cr_debug_sample: kind %u", kind);
    if (!u || !wi || !weight || !valid || ((kind == 1 || kind == 2) && !wo) || (kind == 1 && !param))
        return fail(CR_ERR_INVALID_ARG, "cr_debug_sample: NULL argument");
    Staged a, b, c, o1, o2, o3;
    CR_CUDA(stage_in(a, wo, 12 * (size_t)n, 0));
    CR_CUDA(stage_in(b, u, 8 * (size_t)n, 0));
    CR_CUDA(stage_in(c, param, 16 * (size_t)n, 0));
    CR_CUDA(stage_out(o1, wi, 12 * (size_t)n));
    CR_CUDA(stage_out(o2, weight, 12 * (size_t)n));
    CR_CUDA(stage_out(o3, valid, (size_t)n));
    LaunchCount lc;
    launch_sample(kind, n, static_cast<const float*>(a.dev), static_cast<const float*>(b.dev),
                  static_cast<const float*>(c.dev), static_cast<float*>(o1.dev), static_cast<float*>(o2.dev),
                  static_cast<uint8_t*>(o3.dev), 0, lc);
    CR_CUDA(cudaGetLastError());
    CR_CUDA(finish_out(o1, 0));
    CR_CUDA(finish_out(o2, 0));
    CR_CUDA(finish_out(o3, 0));
    CR_CUDA(cudaStreamSynchronize(0));
    return CR_OK;
}

extern "C" cr_status cr_debug_bvh_check(const float* tri_xyz, uint32_t n_tri, uint32_t flags, cr_bvh_report* rep) {
    g_err.clear();
    if (!tri_xyz || !rep || n_tri == 0 || n_tri > (1u << 28)) return fail(CR_ERR_INVALID_ARG, "cr_debug_bvh_check: bad arguments");
    std::memset(rep, 0, sizeof(*rep));
    try {
        const auto t0 = std::chrono::steady_clock::now();
        const unsigned hc = std::thread::hardware_concurrency();
        HostBVH2 b2 = build_bvh2(tri_xyz, n_tri, hc ? (int)hc : 4);
        const auto t1 = std::chrono::steady_clock::now();
        rep->n_nodes2 = b2.n_nodes;
        rep->depth2 = b2.depth;
        rep->build_ms2 = std::chrono::duration<double, std::milli>(t1 - t0).count();
        check_bvh2(b2, tri_xyz, n_tri, rep->covered2, rep->violations2);
        if (flags & CR_BVH8Q) {
            const auto t2 = std::chrono::steady_clock::now();
            HostBVH8 b8 = build_bvh8q(b2, tri_xyz);
            const auto t3 = std::chrono::steady_clock::now();
            rep->n_nodes8 = b8.n_nodes;
            rep->depth8 = b8.depth;
            rep->stack_bound8 = b8.stack_bound;
            rep->build_ms8 = std::chrono::duration<double, std::milli>(t3 - t2).count();
            check_bvh8(b8, tri_xyz, n_tri, rep->covered8, rep->violations8);
        }
        if (flags & CR_BVH4) {
            HostBVH4 b4 = build_bvh4(b2);
            rep->n_nodes4 = b4.n_nodes;
            rep->depth4 = b4.depth;
            rep->stack_bound4 = b4.stack_bound;
            check_bvh4(b4, b2, tri_xyz, n_tri, rep->covered4, rep->violations4);
        }
    } catch (const std::bad_alloc&) {
        return fail(CR_ERR_OOM, "cr_debug_bvh_check: host allocation");
    }
    return CR_OK;
}

// ------------------------------------------------------------------------------------
// Batches: many jobs in one wavefront, optionally replayed from a CUDA graph.
struct cr_batch {
    std::vector<cr_job> jobs;
    cr_batch_opts opts;
    cr::RenderPlan plan;
    cr::Plan dev;
    cr::Workspace ws;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;
};

static cr_status batch_opts_check(const cr_batch_opts* o, PlanOpts& po, ExecOpts& eo) {
    if (!o) return fail(CR_ERR_INVALID_ARG, "batch options are NULL");
    if (o->bvh != CR_BVH2 && o->bvh != CR_BVH8Q && o->bvh != 0) return fail(CR_ERR_INVALID_ARG, "bvh %u", o->bvh);
    const int block = o->block ? (int)o->block : 128;
    if (block % 32 != 0 || block < 32 || block > 512) return fail(CR_ERR_INVALID_ARG, "block %d", block);
    po.tile_w = o->group_w;
    po.tile_h = o->group_h;
    po.k = o->k;
    po.interleave = o->interleave;
    po.bvh8 = o->bvh == CR_BVH8Q;
    eo.block = block;
    eo.block_secondary = o->block ? block : kSecondaryBlock;
    if (o->stack != 0 && o->stack != 8 && o->stack != 16 && o->stack != 32)
        return fail(CR_ERR_INVALID_ARG, "stack %u not in {8, 16, 32}", o->stack);
    eo.stack = o->stack ? o->stack : 16;
    eo.persistent = (o->flags & CR_OPT_PERSISTENT) != 0;
    eo.ordered_queues = (o->flags & CR_OPT_ORDERED_QUEUES) != 0;
    if (o->sort_key > CR_SORT_HIERARCHY_CUT) return fail(CR_ERR_INVALID_ARG, "sort_key %u", o->sort_key);
    eo.sort_key = o->sort_key;
    return CR_OK;
}

static cr_status check_job_outputs(const cr_job* jobs, uint32_t n) {
    for (uint32_t i = 0; i < n; ++i)
        if (!jobs[i].out_rgb || !is_device_ptr(jobs[i].out_rgb))
            return fail(CR_ERR_INVALID_ARG, "job %u: out_rgb must be a device buffer", i);
    return CR_OK;
}

extern "C" cr_status cr_batch_device_bytes(const cr_job* jobs, uint32_t n_jobs, const cr_batch_opts* opts,
                                           uint64_t* bytes) {
    g_err.clear();
    if (!jobs || !bytes) return fail(CR_ERR_INVALID_ARG, "cr_batch_device_bytes: NULL argument");
    PlanOpts po;
    ExecOpts eo;
    cr_status st = batch_opts_check(opts, po, eo);
    if (st != CR_OK) return st;
    RenderPlan plan;
    st = build_plan(jobs, n_jobs, po, plan);
    if (st != CR_OK) return st;
    *bytes = workspace_bytes(plan.max_slots, plan.npx_total) + sizeof(JobDev) * plan.jobs.size() +
             sizeof(SceneDev) * plan.scenes.size() + (plan.nee ? 48 * (uint64_t)plan.max_slots : 0);
    return CR_OK;
}

extern "C" cr_status cr_batch_create(const cr_job* jobs, uint32_t n_jobs, const cr_batch_opts* opts, cr_batch** out) {
    g_err.clear();
    if (!out || !jobs) return fail(CR_ERR_INVALID_ARG, "cr_batch_create: NULL argument");
    *out = nullptr;
    PlanOpts po;
    ExecOpts eo;
    cr_status st = batch_opts_check(opts, po, eo);
    if (st != CR_OK) return st;
    st = check_job_outputs(jobs, n_jobs);
    if (st != CR_OK) return st;
    std::unique_ptr<cr_batch> b(new (std::nothrow) cr_batch());
    if (!b) return fail(CR_ERR_OOM, "cr_batch_create: host allocation");
    b->jobs.assign(jobs, jobs + n_jobs);
    b->opts = *opts;
    st = build_plan(b->jobs.data(), n_jobs, po, b->plan);
    if (st != CR_OK) return st;
    if (opts->stream) {
        b->stream = static_cast<cudaStream_t>(opts->stream);
    } else {
        CR_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    st = b->ws.ensure(b->plan.max_slots, b->plan.npx_total);
    if (st != CR_OK) return st;
    if (b->plan.nee) {
        st = b->ws.ensure_nee(b->plan.max_slots);
        if (st != CR_OK) return st;
    }
    st = b->dev.upload(b->plan, b->stream);
    if (st != CR_OK) return st;
    CR_CUDA(cudaStreamSynchronize(b->stream));
    if (opts->flags & CR_BATCH_GRAPH) {
        LaunchCount lc;
        CR_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        st = enqueue_plan(b->plan, b->dev, b->ws, eo, b->stream, lc, nullptr);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (st != CR_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(CR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        b->graph = g;
        CR_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
        b->launches = lc.n;
    }
    *out = b.release();
    return CR_OK;
}

extern "C" cr_status cr_batch_run(cr_batch* b, cr_stats* stats) {
    g_err.clear();
    if (!b) return fail(CR_ERR_INVALID_ARG, "cr_batch_run: NULL batch");
    PlanOpts po;
    ExecOpts eo;
    cr_status st = batch_opts_check(&b->opts, po, eo);
    if (st != CR_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stats) {
        CR_CUDA(cudaEventCreate(&e0));
        CR_CUDA(cudaEventCreate(&e1));
        CR_CUDA(cudaEventRecord(e0, b->stream));
    }
    uint64_t launches = b->launches;
    if (b->exec) {
        CR_CUDA(cudaGraphLaunch(b->exec, b->stream));
    } else {
        LaunchCount lc;
        st = enqueue_plan(b->plan, b->dev, b->ws, eo, b->stream, lc, nullptr);
        if (st != CR_OK) return st;
        launches = lc.n;
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        CR_CUDA(cudaEventRecord(e1, b->stream));
        uint64_t host_counts[kCountsWords / 2];
        CR_CUDA(cudaMemcpyAsync(host_counts, b->ws.pb.counts, 4 * kCountsWords, cudaMemcpyDeviceToHost, b->stream));
        CR_CUDA(cudaStreamSynchronize(b->stream));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        stats->ms_total = ms;
        const uint64_t* stat = host_counts + kStatWord / 2;
        for (uint32_t bb = 1; bb <= b->plan.max_bounces; ++bb) stats->secondary_rays += stat[bb];
        stats->secondary_rays_b1 = stat[1];
        stats->shadow_rays = host_counts[kShadowWord / 2];
        uint64_t prim = 0;
        for (const cr_job& j : b->jobs) prim += (uint64_t)j.camera.width * j.camera.height * j.spp;
        stats->primary_rays = prim;
        stats->kernel_launches = launches;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const cr_status qst = queue_status(host_counts);
        if (qst != CR_OK) return qst;
    }
    CR_CUDA(cudaStreamSynchronize(b->stream));
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

extern "C" cr_status cr_batch_destroy(cr_batch* b) {
    g_err.clear();
    if (!b) return CR_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->ws.release();
    b->dev.release();
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return CR_OK;
}

// Quality guard of the autotuner: a reference of the probe job (independent sampling,
// kTuneRefSpp samples from frames no candidate uses) and each grouping's MSE against it.
constexpr uint32_t kTuneRefSpp = 64;
constexpr double kTuneMseMargin = 0.10;

struct TuneProbe {
    bool on = false;
    uint32_t job = 0;
    size_t n = 0;               // floats of the image
    DevMem img;                 // device render target
    std::vector<float> ref, host;
    std::map<uint64_t, double> mse; // by (W, H, K, interleave)
};

static cr_status probe_render(const cr_job& j, uint32_t W, uint32_t H, uint32_t K, uint32_t il, uint32_t spp,
                              uint32_t mode, uint64_t seed, uint32_t frame_base, float* out) {
    cr_render_opts o;
    cr_render_opts_default(&o);
    o.k = K;
    o.interleave = il;
    o.seed = seed;
    o.frame_base = frame_base;
    o.reuse_depth = j.reuse_depth;
    o.diffuse_roughness = j.diffuse_roughness;
    o.flags = ((j.flags & CR_JOB_NEE) ? (uint32_t)CR_OPT_NEE : 0u) |
              ((j.flags & CR_JOB_HYBRID_DONOR) ? (uint32_t)CR_OPT_HYBRID_DONOR : 0u) |
              ((j.flags & CR_JOB_NEE_SHARED) ? (uint32_t)CR_OPT_NEE_SHARED : 0u);
    return cr_render_ex(j.scene, &j.camera, spp, j.max_bounces, (cr_reuse_mode)mode, W, H, out, &o);
}

static cr_status probe_setup(const cr_job* jobs, uint32_t n_jobs, TuneProbe& pr) {
    uint64_t best = 0;
    for (uint32_t i = 0; i < n_jobs; ++i) {
        if (jobs[i].mode != CR_DIRECTION_REUSE && jobs[i].mode != CR_WORLD_REUSE) continue;
        const uint64_t px = (uint64_t)jobs[i].camera.width * jobs[i].camera.height;
        const bool fits = px <= 512ull * 512ull;
        const uint64_t cur = pr.on ? (uint64_t)jobs[pr.job].camera.width * jobs[pr.job].camera.height : 0;
        const bool cur_fits = pr.on && cur <= 512ull * 512ull;
        // the largest job that fits, else the smallest
        if (!pr.on || (fits && (!cur_fits || px > best)) || (!fits && !cur_fits && px < best)) {
            pr.on = true;
            pr.job = i;
            best = px;
        }
    }
    if (!pr.on) return CR_OK;
    const cr_job& j = jobs[pr.job];
    pr.n = 3ull * j.camera.width * j.camera.height;
    CR_CUDA(pr.img.alloc(4 * pr.n));
    float* d = static_cast<float*>(pr.img.p);
    cr_status st = probe_render(j, 8, 8, 8, 1, kTuneRefSpp, CR_INDEPENDENT, j.seed ^ 0x9e3779b97f4a7c15ull,
                                j.frame_base + (1u << 24), d);
    if (st != CR_OK) return st;
    pr.ref.resize(pr.n);
    pr.host.resize(pr.n);
    CR_CUDA(cudaMemcpy(pr.ref.data(), d, 4 * pr.n, cudaMemcpyDeviceToHost));
    return CR_OK;
}

static cr_status probe_mse(const cr_job* jobs, TuneProbe& pr, uint32_t W, uint32_t H, uint32_t K, uint32_t il,
                           double& mse) {
    const uint64_t key = ((uint64_t)W << 48) | ((uint64_t)H << 32) | ((uint64_t)K << 8) | il;
    auto it = pr.mse.find(key);
    if (it != pr.mse.end()) {
        mse = it->second;
        return CR_OK;
    }
    const cr_job& j = jobs[pr.job];
    float* d = static_cast<float*>(pr.img.p);
    cr_status st = probe_render(j, W, H, K, il, j.spp, j.mode, j.seed, j.frame_base, d);
    if (st != CR_OK) return st;
    CR_CUDA(cudaMemcpy(pr.host.data(), d, 4 * pr.n, cudaMemcpyDeviceToHost));
    // MSE of the 4x4-pixel block means: independent pixel errors average down by 16 there,
    // errors correlated within a block (directions shared by neighbouring pixels) do not
    const uint32_t w = j.camera.width, h = j.camera.height;
    double acc = 0.0;
    uint64_t nb = 0;
    for (uint32_t by = 0; by + 4 <= h; by += 4)
        for (uint32_t bx = 0; bx + 4 <= w; bx += 4)
            for (int c = 0; c < 3; ++c) {
                double e = 0.0;
                for (uint32_t y = by; y < by + 4; ++y)
                    for (uint32_t x = bx; x < bx + 4; ++x) {
                        const size_t i = 3 * ((size_t)y * w + x) + c;
                        e += (double)pr.host[i] - (double)pr.ref[i];
                    }
                e /= 16.0;
                acc += e * e;
                ++nb;
            }
    mse = nb ? acc / (double)nb : 0.0;
    pr.mse[key] = mse;
    return CR_OK;
}

extern "C" cr_status cr_batch_autotune(const cr_job* jobs, uint32_t n_jobs, uint32_t allow_contiguous,
                                       cr_batch_opts* opts, cr_tune_report* report) {
    g_err.clear();
    if (!jobs || !opts) return fail(CR_ERR_INVALID_ARG, "cr_batch_autotune: NULL argument");
    cr_tune_report rep;
    std::memset(&rep, 0, sizeof(rep));
    rep.best_ms = 1e30;
    const uint32_t tiles[3][2] = {{4, 4}, {8, 8}, {16, 16}};
    TuneProbe probe;
    {
        cr_status pst = probe_setup(jobs, n_jobs, probe);
        if (pst != CR_OK) return pst;
    }
    if (probe.on) {
        rep.probe_job = probe.job;
        cr_status pst = probe_mse(jobs, probe, 8, 8, 8, 1, rep.default_mse);
        if (pst != CR_OK) return pst;
    }
    auto time_one = [&](const cr_batch_opts& o, double& ms_out) -> cr_status {
        cr_batch* b = nullptr;
        cr_status st = cr_batch_create(jobs, n_jobs, &o, &b);
        if (st != CR_OK) return st;
        cr_stats s1;
        double best = 1e30;
        for (int r = 0; r < 3; ++r) { // one warm-up, best of two
            st = cr_batch_run(b, &s1);
            if (st != CR_OK) break;
            if (r > 0) best = std::min(best, s1.ms_total);
        }
        cr_batch_destroy(b);
        ms_out = best;
        return st;
    };
    for (const auto& t : tiles) {
        const uint32_t m = t[0] * t[1];
        for (uint32_t k = 4; k <= m / 4 && k <= 64; k *= 2) {
            for (uint32_t il_i = 0; il_i < (allow_contiguous ? 2u : 1u); ++il_i) {
                const uint32_t il = 1u - il_i;
                double mse = 0.0;
                if (probe.on) {
                    cr_status pst = probe_mse(jobs, probe, t[0], t[1], k, il, mse);
                    if (pst != CR_OK) return pst;
                }
                const bool rejected = probe.on && mse > rep.default_mse * (1.0 + kTuneMseMargin);
                for (uint32_t block : {64u, 128u, 256u}) {
                    if (rejected) { // not timed: its grouping fails the quality guard
                        rep.n_rejected++;
                        continue;
                    }
                    cr_batch_opts o = *opts;
                    o.group_w = t[0];
                    o.group_h = t[1];
                    o.k = k;
                    o.interleave = il;
                    o.block = block;
                    o.flags &= ~(uint32_t)CR_BATCH_GRAPH;
                    double ms = 0;
                    cr_status st = time_one(o, ms);
                    if (st != CR_OK) return st;
                    rep.n_candidates++;
                    rep.worst_ms = std::max(rep.worst_ms, ms);
                    if (t[0] == 8 && k == 8 && il == 1 && block == 128) rep.default_ms = ms;
                    if (ms < rep.best_ms) {
                        rep.best_mse = mse;
                        rep.best_ms = ms;
                        rep.best_group_w = t[0];
                        rep.best_group_h = t[1];
                        rep.best_k = k;
                        rep.best_interleave = il;
                        rep.best_block = block;
                    }
                }
            }
        }
    }
    // second stage: the stack depth in shared memory for the winner of the first
    rep.best_stack = opts->stack ? opts->stack : 16;
    for (uint32_t stack : {8u, 16u, 32u}) {
        cr_batch_opts o = *opts;
        o.group_w = rep.best_group_w;
        o.group_h = rep.best_group_h;
        o.k = rep.best_k;
        o.interleave = rep.best_interleave;
        o.block = rep.best_block;
        o.stack = stack;
        o.flags &= ~(uint32_t)CR_BATCH_GRAPH;
        double ms = 0;
        cr_status st = time_one(o, ms);
        if (st != CR_OK) return st;
        rep.n_candidates++;
        rep.worst_ms = std::max(rep.worst_ms, ms);
        if (ms < rep.best_ms) {
            rep.best_ms = ms;
            rep.best_stack = stack;
        }
    }
    opts->group_w = rep.best_group_w;
    opts->group_h = rep.best_group_h;
    opts->k = rep.best_k;
    opts->interleave = rep.best_interleave;
    opts->block = rep.best_block;
    opts->stack = rep.best_stack;
    if (report) *report = rep;
    return CR_OK;
}
