// C-ABI entry points of libhuff (declared in include/huff.h): argument checks,
// workspace carving and kernel dispatch.  No compute happens here.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <map>
#include <utility>

#include "kernels.cuh"

namespace huff {

static std::atomic<uint64_t> g_launches{0};

// Launches enqueued while a graph is being captured run only when the graph
// runs; the capturing thread turns counting off and the graph launch counts them.
static thread_local bool t_count_off = false;

void launch_count_suppress(bool on) { t_count_off = on; }

void note_launch(int k) {
    if (!t_count_off) g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed);
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

bool allow_dynamic_smem(const void *func, size_t need) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> limit;   // dynamic bytes allowed per (device, kernel)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lock(mu);
    auto it = limit.find({dev, func});
    if (it == limit.end()) {
        int optin = 0;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || optin <= 0)
            return false;
        // static shared memory of the kernel counts against the same maximum
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, func) != cudaSuccess || fa.sharedSizeBytes > (size_t)optin) return false;
        const int lim = optin - (int)fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) return false;
        it = limit.emplace(std::make_pair(dev, func), lim).first;
    }
    return need <= (size_t)it->second;
}

static bool dtype_ok(huff_dtype d) { return d == HUFF_U8 || d == HUFF_U16 || d == HUFF_U32; }

static bool nbins_ok(huff_dtype d, uint32_t nbins) {
    if (nbins < 1 || nbins > HUFF_MAX_BINS) return false;
    if (d == HUFF_U8 && nbins > 256) return false;
    if (d == HUFF_U16 && nbins > 65536) return false;
    return true;
}

// Typed device arrays must be aligned to their element size.
static bool elem_aligned(const void *p, huff_dtype d) { return ((uintptr_t)p % (uintptr_t)d) == 0; }

static uint32_t *status_of(void *ws) { return static_cast<uint32_t *>(ws); }
static uint8_t *scratch_of(void *ws) { return static_cast<uint8_t *>(ws) + kWsHeaderBytes; }

}  // namespace huff

using namespace huff;

extern "C" {

void huff_default_params(huff_params *p) {
    if (!p) return;
    p->chunk_log2 = 10;
    p->reduce_log2 = -1;
    p->block_threads = 0;
    p->merge = HUFF_MERGE_AUTO;
    p->word_bits = 32;
    p->layout = HUFF_LAYOUT_DENSE;
}

int huff_reduce_factor(double avg_bits, int word_bits) {
    // floor(log2 beta) + r + 1 = log2(word_bits)
    if (!(avg_bits > 0) || word_bits <= 0) return 3;
    int lw = (int)std::lround(std::log2((double)word_bits));
    int r = lw - 1 - (int)std::floor(std::log2(avg_bits));
    if (r < 0) r = 0;
    if (r > lw) r = lw;
    return r;
}

size_t huff_codebook_bytes(uint32_t nbins) {
    return sizeof(huff_codebook_header) + 8ull * nbins + 4ull * nbins;
}

uint64_t huff_max_output_words(uint64_t n, uint32_t max_len) {
    return (n * (uint64_t)max_len + 31) / 32;
}

uint64_t huff_max_output_units(uint64_t n, uint32_t max_len, const huff_params *p) {
    huff_params prm;
    huff_default_params(&prm);
    if (p) prm = *p;
    const uint64_t W = prm.word_bits == 8 ? 8 : prm.word_bits == 16 ? 16 : 32;
    uint64_t u = (n * (uint64_t)max_len + W - 1) / W;
    if (prm.layout == HUFF_LAYOUT_CHUNK_ALIGNED && prm.chunk_log2 >= 0 && prm.chunk_log2 <= 40)
        u += (n + (1ull << prm.chunk_log2) - 1) >> prm.chunk_log2;
    return u;
}

size_t huff_workspace_bytes(uint64_t n, uint32_t nbins, const huff_params *p) {
    size_t a = encode_scratch_bytes(n, nbins);
    if (p && p->merge == HUFF_MERGE_SHUFFLE && p->chunk_log2 >= 4 && p->chunk_log2 <= 30) {
        const size_t b = shuffle_scratch_bytes(n, p->chunk_log2, p->reduce_log2);
        if (b > a) a = b;
    }
    size_t b = codebook_scratch_bytes(nbins);
    size_t s = a > b ? a : b;
    return kWsHeaderBytes + ((s + 255) & ~size_t(255));
}

huff_status huff_workspace_init(void *d_ws, void *stream) {
    if (!d_ws) return HUFF_ERR_INVALID_ARG;
    return cudaMemsetAsync(d_ws, 0, kWsHeaderBytes, (cudaStream_t)stream) == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

huff_status huff_histogram(const void *d_sym, uint64_t n, huff_dtype dtype, uint32_t nbins, uint32_t *d_hist,
                           void *d_ws, void *stream) {
    if (!dtype_ok(dtype) || !nbins_ok(dtype, nbins) || !d_hist || !d_ws || (n && !d_sym) || n >= (1ull << 32))
        return HUFF_ERR_INVALID_ARG;
    if (!elem_aligned(d_sym, dtype) || ((uintptr_t)d_hist & 3) != 0) return HUFF_ERR_INVALID_ARG;
    return histogram_launch(d_sym, n, dtype, nbins, d_hist, status_of(d_ws), (cudaStream_t)stream);
}

huff_status huff_build_codebook(const uint32_t *d_hist, uint32_t nbins, void *d_codebook, void *d_ws, void *stream) {
    if (!d_hist || !d_codebook || !d_ws || nbins < 1 || nbins > HUFF_MAX_BINS) return HUFF_ERR_INVALID_ARG;
    if (((uintptr_t)d_codebook & 15) != 0) return HUFF_ERR_INVALID_ARG;
    return codebook_launch(d_hist, nbins, d_codebook, scratch_of(d_ws), status_of(d_ws), (cudaStream_t)stream);
}

huff_status huff_encode(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook, uint32_t nbins,
                        const huff_params *p, uint32_t *d_out, uint64_t out_capacity_words,
                        uint64_t *d_chunk_bit_offset, uint64_t *d_total_bits, void *d_ws, void *stream) {
    huff_params prm;
    huff_default_params(&prm);
    if (p) prm = *p;
    if (!dtype_ok(dtype) || !nbins_ok(dtype, nbins) || !d_codebook || !d_chunk_bit_offset || !d_total_bits ||
        !d_ws || (n && (!d_sym || !d_out)) || n >= (1ull << 32))
        return HUFF_ERR_INVALID_ARG;
    if (((uintptr_t)d_codebook & 15) != 0) return HUFF_ERR_INVALID_ARG;
    if (!elem_aligned(d_sym, dtype) || ((uintptr_t)d_out & 3) != 0 || ((uintptr_t)d_chunk_bit_offset & 7) != 0 ||
        ((uintptr_t)d_total_bits & 7) != 0)
        return HUFF_ERR_INVALID_ARG;
    if (prm.chunk_log2 < 4 || prm.chunk_log2 > 30 || prm.chunk_log2 < encode_run_log2(dtype)) return HUFF_ERR_INVALID_ARG;
    if (prm.reduce_log2 != -1 && (prm.reduce_log2 < 0 || prm.reduce_log2 > prm.chunk_log2)) return HUFF_ERR_INVALID_ARG;
    if (prm.merge < HUFF_MERGE_AUTO || prm.merge > HUFF_MERGE_SHUFFLE) return HUFF_ERR_INVALID_ARG;
    uint32_t fmt = 0;
    if (encode_format_of(prm, dtype, &fmt) != HUFF_OK) return HUFF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        if (cudaMemsetAsync(d_chunk_bit_offset, 0, 8, st) != cudaSuccess) return HUFF_ERR_CUDA;
        if (cudaMemsetAsync(d_total_bits, 0, 8, st) != cudaSuccess) return HUFF_ERR_CUDA;
        return HUFF_OK;
    }
    if (prm.merge == HUFF_MERGE_SHUFFLE)
        return encode_shuffle_launch(d_sym, n, dtype, d_codebook, nbins, prm.chunk_log2, prm.reduce_log2, 48, d_out,
                                     out_capacity_words, d_chunk_bit_offset, d_total_bits, scratch_of(d_ws),
                                     status_of(d_ws), st);
    return encode_launch(d_sym, n, dtype, d_codebook, nbins, prm.chunk_log2, prm.reduce_log2, fmt, d_out,
                         out_capacity_words, d_chunk_bit_offset, d_total_bits, scratch_of(d_ws), status_of(d_ws), st);
}

huff_status huff_encode_fault_test(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook,
                                   uint32_t nbins, uint32_t *d_out, uint64_t out_capacity_words,
                                   uint64_t *d_chunk_bit_offset, uint64_t *d_total_bits, uint32_t poll_limit,
                                   void *d_ws, void *stream) {
    if (!dtype_ok(dtype) || !nbins_ok(dtype, nbins) || !d_codebook || !d_chunk_bit_offset || !d_total_bits ||
        !d_ws || !d_sym || !d_out || n >= (1ull << 32) || n <= encode_sub_symbols(dtype) * 8ull)   // an encode tile holds at most 8 sub-tiles
        return HUFF_ERR_INVALID_ARG;
    if (poll_limit < 1 || poll_limit > kSpinLimit) return HUFF_ERR_INVALID_ARG;
    if (((uintptr_t)d_codebook & 15) != 0 || !elem_aligned(d_sym, dtype) || ((uintptr_t)d_out & 3) != 0 ||
        ((uintptr_t)d_chunk_bit_offset & 7) != 0 || ((uintptr_t)d_total_bits & 7) != 0)
        return HUFF_ERR_INVALID_ARG;
    huff_params prm;
    huff_default_params(&prm);
    return encode_launch_ex(d_sym, n, dtype, d_codebook, nbins, prm.chunk_log2, prm.reduce_log2, 0u, d_out,
                            out_capacity_words, d_chunk_bit_offset, d_total_bits, scratch_of(d_ws), status_of(d_ws),
                            (cudaStream_t)stream, 1u, poll_limit);
}

static huff_status decode_checked(const void *d_in, uint64_t total_bits, const uint64_t *d_chunk_bit_offset,
                                  const huff_params &prm, uint64_t n, huff_dtype dtype, const void *d_codebook,
                                  uint32_t nbins, void *d_out, void *d_ws, void *stream) {
    if (!dtype_ok(dtype) || !nbins_ok(dtype, nbins) || !d_codebook || !d_ws || (n && (!d_in || !d_out || !d_chunk_bit_offset)))
        return HUFF_ERR_INVALID_ARG;
    if (prm.chunk_log2 < 0 || prm.chunk_log2 > 30) return HUFF_ERR_INVALID_ARG;
    if (!elem_aligned(d_out, dtype) || ((uintptr_t)d_in & 3) != 0 || ((uintptr_t)d_chunk_bit_offset & 7) != 0 ||
        ((uintptr_t)d_codebook & 15) != 0)
        return HUFF_ERR_INVALID_ARG;
    const int W = prm.word_bits == 0 ? 32 : prm.word_bits;
    if (W != 8 && W != 16 && W != 32) return HUFF_ERR_INVALID_ARG;
    if (prm.layout != HUFF_LAYOUT_DENSE && prm.layout != HUFF_LAYOUT_CHUNK_ALIGNED) return HUFF_ERR_INVALID_ARG;
    const uint32_t fmt = (W == 32 ? 0u : W == 16 ? 1u : 2u) | (prm.layout == HUFF_LAYOUT_CHUNK_ALIGNED ? 0x100u : 0u);
    return decode_launch(d_in, total_bits, d_chunk_bit_offset, prm.chunk_log2, fmt, n, dtype, d_codebook, nbins,
                         d_out, status_of(d_ws), (cudaStream_t)stream);
}

huff_status huff_decode(const uint32_t *d_in, uint64_t total_bits, const uint64_t *d_chunk_bit_offset,
                        int chunk_log2, uint64_t n, huff_dtype dtype, const void *d_codebook, uint32_t nbins,
                        void *d_out, void *d_ws, void *stream) {
    huff_params prm;
    huff_default_params(&prm);
    prm.chunk_log2 = chunk_log2;
    return decode_checked(d_in, total_bits, d_chunk_bit_offset, prm, n, dtype, d_codebook, nbins, d_out, d_ws, stream);
}

huff_status huff_decode_ex(const void *d_in, uint64_t total_bits, const uint64_t *d_chunk_bit_offset,
                           const huff_params *p, uint64_t n, huff_dtype dtype, const void *d_codebook,
                           uint32_t nbins, void *d_out, void *d_ws, void *stream) {
    huff_params prm;
    huff_default_params(&prm);
    if (p) prm = *p;
    return decode_checked(d_in, total_bits, d_chunk_bit_offset, prm, n, dtype, d_codebook, nbins, d_out, d_ws, stream);
}

huff_status huff_get_status(const void *d_ws, void *stream) {
    if (!d_ws) return HUFF_ERR_INVALID_ARG;
    uint32_t v = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&v, d_ws, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HUFF_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HUFF_ERR_CUDA;
    return (huff_status)v;
}

const char *huff_status_string(huff_status s) {
    switch (s) {
        case HUFF_OK: return "ok";
        case HUFF_ERR_INVALID_ARG: return "invalid argument";
        case HUFF_ERR_SYMBOL_RANGE: return "symbol out of range";
        case HUFF_ERR_NOT_IN_CODEBOOK: return "symbol has no codeword";
        case HUFF_ERR_CAPACITY: return "output capacity exceeded";
        case HUFF_ERR_OOM: return "out of memory";
        case HUFF_ERR_TIMEOUT: return "device wait timed out";
        case HUFF_ERR_BUSY: return "busy";
        case HUFF_ERR_CUDA: return "CUDA error";
        case HUFF_ERR_HIST_OVERFLOW: return "histogram sum >= 2^32";
        case HUFF_ERR_NOT_FOUND: return "unknown ticket";
        case HUFF_ERR_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

uint64_t huff_launch_count(void) { return g_launches.load(); }

}  // extern "C"
