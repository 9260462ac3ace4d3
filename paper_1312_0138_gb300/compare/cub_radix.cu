// cub_radix.cu -- comparison point for the benchmark only: the same keys
// sorted by the CUDA toolkit's cub::DeviceRadixSort::SortKeys on the same GPU.
// Not part of the sort library (libbitsort.so never links it); built into a
// separate libcubcompare.so that bench.py loads.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cub/device/device_radix_sort.cuh>

static void *g_temp = nullptr;
static size_t g_temp_bytes = 0;

// Sort n uint32 keys (device pointers, keys and out distinct) on bits
// [0, end_bit) on `stream`.  Returns a cudaError_t value.
extern "C" int cub_radix_sort_keys(const uint32_t *keys, uint32_t *out, uint64_t n, int end_bit, void *stream) {
    size_t need = 0;
    cudaError_t e = cub::DeviceRadixSort::SortKeys(nullptr, need, keys, out, (int64_t)n, 0, end_bit,
                                                   reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return (int)e;
    if (need > g_temp_bytes) {
        if (g_temp) cudaFree(g_temp);
        g_temp = nullptr;
        g_temp_bytes = 0;
        e = cudaMalloc(&g_temp, need);
        if (e != cudaSuccess) return (int)e;
        g_temp_bytes = need;
    }
    e = cub::DeviceRadixSort::SortKeys(g_temp, need, keys, out, (int64_t)n, 0, end_bit,
                                       reinterpret_cast<cudaStream_t>(stream));
    return (int)e;
}
