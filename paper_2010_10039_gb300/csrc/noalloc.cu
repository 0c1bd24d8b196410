// huff_encode_noalloc: the encode of huff_encode for callers that cannot
// allocate device memory at all -- for example a plugin inside a host program
// whose framework owns every device allocation, or a latency-critical loop
// where cudaMalloc/cudaFree (which may synchronise the device) are not
// allowed.  The encoder's scratch (a tile counter and one 16-byte look-back
// descriptor per tile) lives in a fixed array in this file instead of a
// caller workspace.
#include <mutex>

#include "kernels.cuh"

namespace huff {

// Largest input of one call, and the encoder scratch it needs: a tile counter
// and a 16-byte descriptor per tile of >= 2048 symbols (2 MiB + 64 bytes,
// rounded up to 256), then room for the 32-bit table entries of the largest
// alphabet (256 KiB).
constexpr uint64_t kNoAllocMaxSymbols = 1ull << 28;
constexpr size_t kNoAllocScratchBytes =
    ((64 + 16 * (kNoAllocMaxSymbols / 2048) + 255) & ~size_t(255)) + 4ull * HUFF_MAX_BINS_BATCH;

// One copy per device that loads the library; it stays until the process exits.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static uint8_t *g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of the array on the current device.  Outside a stream
// capture it is looked up on every call, so a call after cudaDeviceReset (a
// new primary context, the module loaded again) gets the new address.  While
// `st` is being captured no lookup is made -- it could load the module inside
// the capture -- and the address of the last uncaptured call on this device
// is used; the first call on a device must therefore come before any capture.
static uint8_t *noalloc_scratch(cudaStream_t st, huff_status *err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        *err = HUFF_ERR_CUDA;
        return nullptr;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        *err = HUFF_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            *err = HUFF_ERR_CUDA;
            return nullptr;
        }
        g_scratch_addr[dev] = static_cast<uint8_t *>(ptr);
    } else if (!g_scratch_addr[dev]) {
        *err = HUFF_ERR_INVALID_ARG;          // first call on this device inside a capture
        return nullptr;
    }
    return g_scratch_addr[dev];
}

}  // namespace huff

using namespace huff;

extern "C" huff_status huff_encode_noalloc(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook,
                                           uint32_t nbins, const huff_params *p, uint32_t *d_out,
                                           uint64_t out_capacity_words, uint64_t *d_chunk_bit_offset,
                                           uint64_t *d_total_bits, uint32_t *d_status, void *stream) {
    huff_params prm;
    huff_default_params(&prm);
    if (p) prm = *p;
    if (n > kNoAllocMaxSymbols) return HUFF_ERR_INVALID_ARG;          // beyond the fixed scratch
    if (!d_status || !d_codebook || !d_chunk_bit_offset || !d_total_bits || (n && (!d_sym || !d_out)))
        return HUFF_ERR_INVALID_ARG;
    if (dtype != HUFF_U8 && dtype != HUFF_U16 && dtype != HUFF_U32) return HUFF_ERR_INVALID_ARG;
    if (nbins < 1 || nbins > HUFF_MAX_BINS_BATCH || (dtype == HUFF_U8 && nbins > 256)) return HUFF_ERR_INVALID_ARG;
    if (((uintptr_t)d_codebook & 15) != 0) return HUFF_ERR_INVALID_ARG;
    if (((uintptr_t)d_sym % (uintptr_t)dtype) != 0 || ((uintptr_t)d_out & 3) != 0 ||
        ((uintptr_t)d_chunk_bit_offset & 7) != 0 || ((uintptr_t)d_total_bits & 7) != 0 || ((uintptr_t)d_status & 3) != 0)
        return HUFF_ERR_INVALID_ARG;
    if (prm.chunk_log2 < 4 || prm.chunk_log2 > 30 || prm.chunk_log2 < encode_run_log2(dtype)) return HUFF_ERR_INVALID_ARG;
    if (prm.reduce_log2 != -1 && (prm.reduce_log2 < 0 || prm.reduce_log2 > prm.chunk_log2)) return HUFF_ERR_INVALID_ARG;
    // the fixed array is sized for the fused encoder only: the paper-layout
    // merge (HUFF_MERGE_SHUFFLE) needs chunk slots it does not have
    if (prm.merge != HUFF_MERGE_AUTO && prm.merge != HUFF_MERGE_SCAN) return HUFF_ERR_INVALID_ARG;
    uint32_t fmt = 0;
    if (encode_format_of(prm, dtype, &fmt) != HUFF_OK) return HUFF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    huff_status err = HUFF_OK;
    uint8_t *scratch = noalloc_scratch(st, &err);
    if (!scratch) return err;
    if (cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st) != cudaSuccess) return HUFF_ERR_CUDA;
    if (n == 0) {
        if (cudaMemsetAsync(d_chunk_bit_offset, 0, 8, st) != cudaSuccess) return HUFF_ERR_CUDA;
        if (cudaMemsetAsync(d_total_bits, 0, 8, st) != cudaSuccess) return HUFF_ERR_CUDA;
        return HUFF_OK;
    }
    // the encoder clears the part of the scratch it uses before its launch
    if (encode_scratch_bytes(n, nbins) > kNoAllocScratchBytes) return HUFF_ERR_INVALID_ARG;
    return encode_launch(d_sym, n, dtype, d_codebook, nbins, prm.chunk_log2, prm.reduce_log2, fmt, d_out,
                         out_capacity_words, d_chunk_bit_offset, d_total_bits, scratch, d_status, st);
}
