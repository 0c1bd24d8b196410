// Device-side copy of the seeded symbol generator of synth.py, for inputs too
// large to draw on the host (the 3 GB batched workload, served requests made
// on the device).  It holds no Huffman arithmetic and is not part of libhuff:
// it is a separate library used by the benchmark and the tests, and the tests
// check it bit for bit against synth.py.
//
//   mix64(z)          SplitMix64 output finaliser (Steele, Lea & Flood 2014)
//   key(seed, s)      mix64((seed + 1) * G) ^ mix64((s + 1) * K)
//   u64(seed, s, i)   mix64(key(seed, s) + (i + 1) * G)
//   symbol            min{k : (u64 >> 32) < T[k]}, renamed through map[] if given
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kG = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kK = 0xD1B54A32D192ED03ull;
constexpr uint32_t kSmemEntries = 4096;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// first k in [0, K) with u < T[k] (T nondecreasing, T[K-1] = 2^32 > u)
__device__ __forceinline__ uint32_t upper(const uint64_t *T, uint32_t K, uint64_t u) {
    uint32_t lo = 0, hi = K - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (u < T[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

template <typename Sym>
__global__ void __launch_bounds__(256) draw_kernel(Sym *out, uint64_t n, const uint64_t *T, uint32_t K,
                                                   const uint32_t *map, uint64_t key, uint64_t start) {
    __shared__ uint64_t sT[kSmemEntries];
    const bool small = K <= kSmemEntries;
    if (small)
        for (uint32_t i = threadIdx.x; i < K; i += blockDim.x) sT[i] = T[i];
    __syncthreads();
    const uint64_t *tab = small ? sT : T;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t u = mix64(key + (start + i + 1) * kG) >> 32;
        uint32_t k = upper(tab, K, u);
        if (map) k = map[k];
        out[i] = (Sym)k;
    }
}

}  // namespace

extern "C" {

// n symbols of `width` bytes (1, 2, 4) into d_out: element i is the draw for
// index start + i of stream `stream` under `seed`.  d_table: K uint64 (device),
// d_map: K uint32 or NULL.  Returns 0, or a cudaError_t value.
int synth_draw(void *d_out, uint64_t n, int width, const uint64_t *d_table, uint32_t K, const uint32_t *d_map,
               uint64_t seed, uint64_t stream, uint64_t start, void *cuda_stream) {
    if (n == 0) return 0;
    if (!d_out || !d_table || K < 1 || (width != 1 && width != 2 && width != 4)) return (int)cudaErrorInvalidValue;
    const uint64_t key = mix64((seed + 1) * kG) ^ mix64((stream + 1) * kK);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t grid = (n + 255) / 256;
    if (grid > (uint64_t)sms * 16) grid = (uint64_t)sms * 16;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (width == 1) draw_kernel<uint8_t><<<(unsigned)grid, 256, 0, st>>>((uint8_t *)d_out, n, d_table, K, d_map, key, start);
    else if (width == 2) draw_kernel<uint16_t><<<(unsigned)grid, 256, 0, st>>>((uint16_t *)d_out, n, d_table, K, d_map, key, start);
    else draw_kernel<uint32_t><<<(unsigned)grid, 256, 0, st>>>((uint32_t *)d_out, n, d_table, K, d_map, key, start);
    return (int)cudaGetLastError();
}

}  // extern "C"
