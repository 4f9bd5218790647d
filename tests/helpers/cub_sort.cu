// Test helper: CUB's DeviceRadixSort on the same keys as the library's ray sort, as an
// independent cross-check of the sorted order and a timing reference (not product code).
#include <cub/device/device_radix_sort.cuh>
#include <cuda_runtime.h>

#include <cstdint>

extern "C" int cub_sort_pairs(const uint32_t* keys_in, const int32_t* vals_in, uint32_t* keys_out, int32_t* vals_out,
                              uint32_t n, int end_bit, int reps, float* ms) {
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    if (cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, vals_in, vals_out, (int)n, 0, end_bit) !=
        cudaSuccess)
        return 1;
    if (cudaMalloc(&tmp, tmp_bytes) != cudaSuccess) return 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, vals_in, vals_out, (int)n, 0, end_bit);
    cudaEventRecord(e0, 0);
    for (int r = 0; r < reps; ++r)
        cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, vals_in, vals_out, (int)n, 0, end_bit);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float el = 0.0f;
    cudaEventElapsedTime(&el, e0, e1);
    *ms = el / reps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(tmp);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
