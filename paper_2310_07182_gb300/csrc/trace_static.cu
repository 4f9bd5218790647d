// trace_static.cu -- closest-hit tracing that allocates nothing.
//
// cr_trace_rays stages its rays and hits through device buffers it allocates per call.
// Some callers cannot allow that: a host framework that owns all device memory through its
// own pool allocator and forbids raw cudaMalloc, a latency-critical loop that cannot afford
// the implicit device synchronisation of cudaMalloc/cudaFree, or a process that has already
// reserved nearly all device memory so an allocation could fail mid-frame.  For them this
// file keeps the trace kernel's scratch (ray origin/direction records and hit records for up
// to CR_TRACE_STATIC_MAX_RAYS rays, 40 bytes each) in one file-scope __device__ array.  Every
// GPU that loads the library holds that array until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "cr_internal.h"

namespace cr {
namespace {

constexpr size_t kStaticRays = CR_TRACE_STATIC_MAX_RAYS;
constexpr size_t kOffRayO = 0;                       // float4 per ray
constexpr size_t kOffRayD = kOffRayO + 16 * kStaticRays; // float4 per ray
constexpr size_t kOffHit = kOffRayD + 16 * kStaticRays;  // int2 per ray
constexpr size_t kStaticBytes = kOffHit + 8 * kStaticRays;

static __device__ __align__(256) unsigned char g_trace_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_trace_scratch on the current device, looked up once per device.  In
// host code the symbol is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with that device current.
cudaError_t scratch_on_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_trace_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Device (or managed) memory of device `dev`: another GPU's memory is rejected too, since the
// kernels run on the current device.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

} // namespace
} // namespace cr

extern "C" cr_status cr_trace_rays_static(cr_scene* scene, const float* rays, const int32_t* skip_prim, uint32_t n,
                                          int32_t* prim, float* t, void* stream) {
    using namespace cr;
    char msg[256];
    set_last_error("");
    if (!scene) {
        set_last_error("cr_trace_rays_static: scene is NULL");
        return CR_ERR_INVALID_ARG;
    }
    if (n == 0) return CR_OK;
    if (n > kStaticRays) {
        snprintf(msg, sizeof(msg), "cr_trace_rays_static: n=%u exceeds the static scratch of %u rays", n,
                 (unsigned)kStaticRays);
        set_last_error(msg);
        return CR_ERR_INVALID_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cr_trace_rays_static: no current CUDA device");
        return CR_ERR_CUDA;
    }
    if (scene_device(scene) != dev) {
        snprintf(msg, sizeof(msg), "cr_trace_rays_static: the scene lives on device %d, device %d is current",
                 scene_device(scene), dev);
        set_last_error(msg);
        return CR_ERR_INVALID_ARG;
    }
    if (!rays || !prim || !t || !on_device(rays, dev) || !on_device(prim, dev) || !on_device(t, dev) ||
        (skip_prim && !on_device(skip_prim, dev))) {
        set_last_error("cr_trace_rays_static: rays, skip_prim, prim and t must be device pointers of the current device");
        return CR_ERR_INVALID_ARG;
    }
    void* base = nullptr;
    cudaError_t e = scratch_on_current_device(&base);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "cr_trace_rays_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        set_last_error(msg);
        return CR_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* b = static_cast<unsigned char*>(base);
    float4* ro = reinterpret_cast<float4*>(b + kOffRayO);
    float4* rd = reinterpret_cast<float4*>(b + kOffRayD);
    int2* hit = reinterpret_cast<int2*>(b + kOffHit);
    const DevScene& ds = *dev_scene_of(scene);
    LaunchCount lc;
    // the scene's device table entry was made by cr_scene_create, so nothing is allocated here
    // every scratch record read below is written first by this call, so nothing needs clearing
    launch_rays_from_user(rays, skip_prim, n, ro, rd, st, lc);
    TraceArgs ta;
    ta.ray_o = ro;
    ta.ray_d = rd;
    ta.hit = hit;
    ta.n_max = n;
    ta.block = 128;
    ta.scenes = dev_scene_entry(scene, false);
    launch_trace(ta, st, lc);
    launch_hits_to_user(ds.tris, hit, n, prim, t, st, lc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "cr_trace_rays_static: %s", cudaGetErrorString(e));
        set_last_error(msg);
        return CR_ERR_CUDA;
    }
    return CR_OK;
}
