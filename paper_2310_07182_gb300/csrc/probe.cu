// probe.cu -- read-bandwidth probe for the L2 roof of the roofline (cr_measure_l2_read).
#include <cuda_runtime.h>

#include <cstdint>

#include "cr_internal.h"

namespace cr {
namespace {

__global__ void __launch_bounds__(256) k_read(const uint4* __restrict__ buf, size_t n, uint32_t* __restrict__ sink) {
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint4 v = __ldg(&buf[i]);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    // one word per block keeps the loads alive
    acc = __reduce_xor_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31u) == 0 && acc == 0x9e3779b9u) sink[blockIdx.x] = acc;
}

__global__ void k_fill(uint4* __restrict__ buf, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        buf[i] = make_uint4((uint32_t)i, (uint32_t)(i >> 7), 3u, 5u);
}

} // namespace
} // namespace cr

extern "C" cr_status cr_measure_l2_read(uint64_t bytes, uint32_t reps, double* gbs) {
    using namespace cr;
    set_last_error("");
    if (!gbs || reps == 0 || bytes < (1u << 20)) {
        set_last_error("cr_measure_l2_read: bytes >= 1 MiB, reps >= 1 and gbs required");
        return CR_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)(bytes / 16);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t grid = (uint32_t)(sms > 0 ? sms : 1) * 8u;
    void* buf = nullptr;
    void* sink = nullptr;
    if (cudaMalloc(&buf, n * 16) != cudaSuccess || cudaMalloc(&sink, 4 * (size_t)grid) != cudaSuccess) {
        cudaGetLastError();
        if (buf) cudaFree(buf);
        set_last_error("cr_measure_l2_read: device allocation failed");
        return CR_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fill<<<grid, 256>>>(static_cast<uint4*>(buf), n);
    k_read<<<grid, 256>>>(static_cast<const uint4*>(buf), n, static_cast<uint32_t*>(sink));
    cudaEventRecord(e0);
    for (uint32_t r = 0; r < reps; ++r)
        k_read<<<grid, 256>>>(static_cast<const uint4*>(buf), n, static_cast<uint32_t*>(sink));
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    if (e != cudaSuccess || !(ms > 0.0f)) {
        set_last_error("cr_measure_l2_read: CUDA error");
        return CR_ERR_CUDA;
    }
    *gbs = (double)n * 16.0 * reps / (ms * 1e-3) / 1e9;
    return CR_OK;
}
