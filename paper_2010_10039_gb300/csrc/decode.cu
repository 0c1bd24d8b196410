// Treeless canonical decoding (Sec. IV-B2): a codeword of length l is the
// first l-bit window v with v >= First[l]; its symbol is
// sorted_syms[Entry[l] + v - First[l]].  The chunk offsets written by the
// encoder let every chunk be decoded independently: one thread per chunk,
// reading the stream through a 64-bit window.
#include "kernels.cuh"

namespace huff {

constexpr int kDecThreads = 128;

struct DecArgs {
    const uint32_t *in;
    uint64_t total_bits;
    uint64_t in_words;
    const uint64_t *offs;
    int chunk_log2;
    uint64_t n;
    uint64_t nchunks;
    const uint8_t *book;
    uint8_t *out;
    int width;
    uint32_t nbins;
    uint32_t *status;
};

__device__ __forceinline__ uint64_t window64(const uint32_t *in, uint64_t nwords, uint64_t p) {
    uint64_t w = p >> 5;
    uint32_t sh = p & 31;
    uint64_t a = w < nwords ? in[w] : 0, b = w + 1 < nwords ? in[w + 1] : 0, c = w + 2 < nwords ? in[w + 2] : 0;
    uint64_t hi = (a << 32) | b;
    return sh ? (hi << sh) | (c >> (32 - sh)) : hi;
}

__global__ void __launch_bounds__(kDecThreads) decode_kernel(DecArgs a) {
    __shared__ uint64_t s_first[HUFF_MAX_LEN + 1];
    __shared__ uint32_t s_entry[HUFF_MAX_LEN + 1];
    __shared__ uint32_t s_count[HUFF_MAX_LEN + 1];
    const huff_codebook_header *hdr = reinterpret_cast<const huff_codebook_header *>(a.book);
    const uint32_t *sorted_syms = reinterpret_cast<const uint32_t *>(a.book + cb_sorted_offset(a.nbins));
    for (int l = threadIdx.x; l <= HUFF_MAX_LEN; l += blockDim.x) {
        s_first[l] = hdr->first[l];
        s_entry[l] = hdr->entry[l];
        s_count[l] = hdr->count[l];
    }
    __syncthreads();
    const uint32_t max_len = hdr->max_len;
    const uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (c >= a.nchunks) return;
    if (hdr->nbins != a.nbins || max_len == 0 || max_len > HUFF_MAX_LEN) { set_error(a.status, HUFF_ERR_INVALID_ARG); return; }
    uint64_t i0 = c << a.chunk_log2;
    uint64_t i1 = i0 + (1ull << a.chunk_log2);
    if (i1 > a.n) i1 = a.n;
    uint64_t p = a.offs[c];
    const uint64_t pend = a.offs[c + 1];
    for (uint64_t i = i0; i < i1; i++) {
        uint64_t win = window64(a.in, a.in_words, p);
        uint32_t l = 1;
        uint64_t v = 0;
        for (; l <= max_len; l++) {
            v = win >> (64 - l);
            if (v >= s_first[l]) break;
        }
        uint32_t s = 0;
        if (l > max_len || v - s_first[l] >= s_count[l] || p + l > pend) {
            set_error(a.status, HUFF_ERR_INVALID_ARG);
            return;
        }
        s = sorted_syms[s_entry[l] + (uint32_t)(v - s_first[l])];
        p += l;
        if (a.width == 1) a.out[i] = (uint8_t)s;
        else if (a.width == 2) reinterpret_cast<uint16_t *>(a.out)[i] = (uint16_t)s;
        else reinterpret_cast<uint32_t *>(a.out)[i] = s;
    }
    if (p != pend) set_error(a.status, HUFF_ERR_INVALID_ARG);
}

huff_status decode_launch(const uint32_t *d_in, uint64_t total_bits, const uint64_t *d_offs, int chunk_log2,
                          uint64_t n, huff_dtype dtype, const void *d_codebook, uint32_t nbins, void *d_out,
                          uint32_t *status, cudaStream_t st) {
    DecArgs a;
    a.in = d_in;
    a.total_bits = total_bits;
    a.in_words = (total_bits + 31) / 32;
    a.offs = d_offs;
    a.chunk_log2 = chunk_log2;
    a.n = n;
    a.nchunks = (n + (1ull << chunk_log2) - 1) >> chunk_log2;
    a.book = static_cast<const uint8_t *>(d_codebook);
    a.out = static_cast<uint8_t *>(d_out);
    a.width = (int)dtype;
    a.nbins = nbins;
    a.status = status;
    if (a.nchunks == 0) return HUFF_OK;
    uint64_t grid = (a.nchunks + kDecThreads - 1) / kDecThreads;
    decode_kernel<<<(unsigned)grid, kDecThreads, 0, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

}  // namespace huff
