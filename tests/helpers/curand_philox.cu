// Test helper: cuRAND's Philox4_32_10 generator, used only to pin the oracle's Philox.
// With curand_init(seed, subsequence, offset) the generator's key is the seed and its
// 128-bit counter starts at (offset/4 in words 0-1) + (subsequence in words 2-3); curand4
// returns the block for the current counter.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_curand_philox(uint64_t seed, const uint32_t* ctr, uint32_t n, uint32_t* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    const unsigned long long sub = ((unsigned long long)ctr[4 * i + 3] << 32) | ctr[4 * i + 2];
    const unsigned long long off = (((unsigned long long)ctr[4 * i + 1] << 32) | ctr[4 * i + 0]) * 4ull;
    curand_init(seed, sub, off, &st);
    const uint4 r = curand4(&st);
    out[4 * i + 0] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

extern "C" int curand_philox_blocks(uint64_t seed, const uint32_t* ctr_host, uint32_t n, uint32_t* out_host) {
    uint32_t *dc = nullptr, *dout = nullptr;
    if (cudaMalloc(&dc, 16ull * n) != cudaSuccess) return 1;
    if (cudaMalloc(&dout, 16ull * n) != cudaSuccess) return 2;
    cudaMemcpy(dc, ctr_host, 16ull * n, cudaMemcpyHostToDevice);
    k_curand_philox<<<(n + 127) / 128, 128>>>(seed, dc, n, dout);
    cudaError_t e = cudaMemcpy(out_host, dout, 16ull * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    return e == cudaSuccess ? 0 : 3;
}
