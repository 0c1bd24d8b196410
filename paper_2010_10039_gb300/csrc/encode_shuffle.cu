// Encoding as laid out in the paper (Sec. IV-C with the gathering of Table I),
// selected by huff_params.merge = HUFF_MERGE_SHUFFLE; the default path is the
// fused single-pass kernel of encode_impl.cuh.  Same output, three kernels:
//
//  1. reduce-shuffle-merge, one CTA per chunk of N = 2^M symbols, 2^s threads
//     (s = M - r): thread i concatenates the codewords of symbols
//     [i 2^r, (i+1) 2^r) of the chunk (reduce-merge, Merge((a,l)_{2k},
//     (a,l)_{2k+1}) = (a_{2k} (+) a_{2k+1}, l_{2k} + l_{2k+1})) into its slot
//     of shared memory; then s log steps: at step k the groups of 2^k threads
//     append their right half's bits after their left half's bits
//     (shuffle-merge), until the chunk is one dense run; the run goes to a
//     chunk-aligned slot of global scratch with its bit length;
//  2. an exclusive scan of the chunk lengths gives the chunk bit offsets and
//     total_bits ("get blockwise code len" + prefix sum);
//  3. the coalescing copy: every chunk writes the stream words whose last bit
//     it holds (the first such word also takes the tail bits of the chunks
//     before it), so every word is written once with plain stores.
//
// Unlike the paper, a thread's merged run may be longer than a word: slots
// hold up to 2^r * max_len bits, so no codeword is broken off ("breaking").
#include "kernels.cuh"

namespace huff {

constexpr int kShufMaxThreads = 1024;
constexpr int kShufMaxR = 4;               // 2^r <= 16 symbols per thread
constexpr int kShufMaxLen = 48;            // slots are sized for codewords of up to 48 bits
// destination words one thread moves in one step: at most ceil((h Q + 1) / 2h) <= Q / 2 + 1
constexpr int kShufMaxPer = ((1 << kShufMaxR) * kShufMaxLen / 32 + 2) / 2 + 2;
constexpr int kScanThreads = 1024;

struct ShufArgs {
    const uint8_t *sym;
    uint64_t n;
    const uint64_t *cw;        // codebook codewords (len << 58 | code)
    uint32_t nbins;
    int M;                     // chunk = 2^M symbols
    int r;                     // 2^r symbols per thread
    uint32_t slot_words;       // words per thread slot: ceil(2^r * max_len / 32)
    uint32_t *scratch;         // chunk c at c * (2^(M-r) * slot_words) words
    uint64_t *chunk_bits;      // bit length of every chunk
    uint32_t *status;
};

// Appends l (<= 64) bits to a shared-memory bit string at bit position pos
// (bits after pos are zero), one word at a time.
__device__ __forceinline__ void put_bits(uint32_t *buf, uint32_t pos, uint64_t code, uint32_t l) {
    while (l) {
        const uint32_t w = pos >> 5, off = pos & 31, room = 32 - off;
        const uint32_t take = l < room ? l : room;
        const uint32_t part = (uint32_t)(code >> (l - take)) & (take == 32 ? 0xFFFFFFFFu : ((1u << take) - 1));
        buf[w] |= part << (room - take);
        pos += take;
        l -= take;
    }
}

template <typename Sym>
__global__ void __launch_bounds__(kShufMaxThreads) shuffle_merge_kernel(ShufArgs a) {
    extern __shared__ uint32_t sbuf[];           // 2^s slots of slot_words
    __shared__ uint32_t len[kShufMaxThreads];    // bit length of every group's run
    const uint32_t T = blockDim.x, i = threadIdx.x;
    const uint32_t Q = a.slot_words;
    const uint64_t c = blockIdx.x;
    const uint64_t chunk0 = c << a.M;
    const Sym *sp = reinterpret_cast<const Sym *>(a.sym);
    // the codebook must be the alphabet the caller names (cw[] is read up to nbins)
    if (reinterpret_cast<const huff_codebook_header *>(reinterpret_cast<const uint8_t *>(a.cw) - cb_cw_offset())->nbins !=
        a.nbins) {
        if (i == 0) set_error(a.status, HUFF_ERR_INVALID_ARG);
        return;
    }

    // ---- reduce-merge: thread i's 2^r codewords into its slot
    uint32_t *mine = sbuf + i * Q;
    for (uint32_t k = 0; k < Q; k++) mine[k] = 0;
    uint32_t bits = 0, bad = 0;
    const uint64_t s0 = chunk0 + ((uint64_t)i << a.r);
    for (uint32_t x = 0; x < (1u << a.r); x++) {
        const uint64_t idx = s0 + x;
        if (idx >= a.n) break;
        const uint32_t s = (uint32_t)sp[idx];
        const uint64_t e = s < a.nbins ? __ldg(a.cw + s) : 0ull;
        const uint32_t l = (uint32_t)(e >> HUFF_CW_LEN_SHIFT);
        if (!l) { bad = s < a.nbins ? HUFF_ERR_NOT_IN_CODEBOOK : HUFF_ERR_SYMBOL_RANGE; continue; }
        if (bits + l > (Q - 1) * 32) { bad = HUFF_ERR_INVALID_ARG; continue; }   // longer than the slot allows
        put_bits(mine, bits, e & ((1ull << HUFF_CW_LEN_SHIFT) - 1), l);
        bits += l;
    }
    if (bad) set_error(a.status, bad);
    len[i] = bits;
    __syncthreads();

    // ---- shuffle-merge: s log steps of pairwise group concatenation.  In a
    // group of 2h threads the right half's run (at slot g + h) is appended at
    // bit Ll of the left half's run (at slot g): destination word d0 + q is
    // built from source words q - 1 and q, so every destination word is
    // written whole by one thread and the first one keeps the left tail bits.
    for (uint32_t h = 1; h < T; h <<= 1) {
        const uint32_t g = i & ~(2 * h - 1), j = i - g;
        const uint32_t Ll = len[g], Lr = len[g + h];
        const uint32_t *src = sbuf + (g + h) * Q;
        uint32_t *dst = sbuf + g * Q;
        const uint32_t rw = (Lr + 31) / 32, sh = Ll & 31, d0 = Ll >> 5;
        const uint32_t nd = rw + (sh ? 1 : 0);                        // destination words
        uint32_t va[kShufMaxPer], vb[kShufMaxPer];
        uint32_t nv = 0;
        for (uint32_t q = j; q < nd && nv < kShufMaxPer; q += 2 * h, nv++) {
            va[nv] = (q >= 1 && q - 1 < rw) ? src[q - 1] : 0u;
            vb[nv] = q < rw ? src[q] : 0u;
        }
        __syncthreads();
        nv = 0;
        for (uint32_t q = j; q < nd && nv < kShufMaxPer; q += 2 * h, nv++) {
            uint32_t v;
            if (sh == 0) v = vb[nv];
            else v = (va[nv] << (32 - sh)) | (vb[nv] >> sh);
            if (q == 0 && sh) v |= dst[d0] & (0xFFFFFFFFu << (32 - sh));   // the left half's tail bits
            dst[d0 + q] = v;
        }
        __syncthreads();
        if (j == 0) len[g] = Ll + Lr;
        // the right half's old words past the new end are cleared before the next step
        const uint32_t new_words = (Ll + Lr + 31) / 32, cap = 2 * h * Q;
        for (uint32_t w = new_words + j; w < cap; w += 2 * h) dst[w] = 0;
        __syncthreads();
    }

    // ---- the chunk's dense run to its scratch slot
    const uint32_t L = len[0];
    uint32_t *out = a.scratch + c * (uint64_t)(T * Q);
    for (uint32_t w = i; w < (L + 31) / 32; w += T) out[w] = sbuf[w];
    if (i == 0) a.chunk_bits[c] = L;
}

// Exclusive scan of the chunk lengths (one CTA): chunk bit offsets and total.
__global__ void __launch_bounds__(kScanThreads) chunk_scan_kernel(const uint64_t *chunk_bits, uint64_t nchunks,
                                                                 uint64_t *offs, uint64_t *total) {
    __shared__ uint64_t part[kScanThreads];
    const uint32_t i = threadIdx.x;
    const uint64_t per = (nchunks + kScanThreads - 1) / kScanThreads;
    const uint64_t b = i * per, e = b + per < nchunks ? b + per : nchunks;
    uint64_t sum = 0;
    for (uint64_t c = b; c < e; c++) sum += chunk_bits[c];
    part[i] = sum;
    __syncthreads();
    for (uint32_t o = 1; o < kScanThreads; o <<= 1) {
        const uint64_t y = i >= o ? part[i - o] : 0;
        __syncthreads();
        part[i] += y;
        __syncthreads();
    }
    uint64_t run = part[i] - sum;
    for (uint64_t c = b; c < e; c++) {
        offs[c] = run;
        run += chunk_bits[c];
    }
    if (i == kScanThreads - 1) {
        offs[nchunks] = part[i];
        *total = part[i];
    }
}

// Bits [b, b + 32) of the stream as one word, read from the chunk scratch
// slots (bits past the end are zero).  Walks forward from chunk k, which
// holds bit b.
__device__ uint32_t stream_word(const uint32_t *scratch, uint64_t slot, const uint64_t *offs, uint64_t nchunks,
                                uint64_t k, uint64_t b) {
    uint32_t word = 0, have = 0;
    while (have < 32 && k < nchunks) {
        const uint64_t cb = offs[k], ce = offs[k + 1];
        if (b + have >= ce) { k++; continue; }
        const uint64_t rel = b + have - cb;                      // bit inside chunk k
        const uint32_t *ch = scratch + k * slot;
        const uint32_t w = (uint32_t)(rel >> 5), o = (uint32_t)(rel & 31);
        uint64_t pair = ((uint64_t)ch[w] << 32);
        if ((uint64_t)(w + 1) * 32 < ce - cb) pair |= ch[w + 1];
        const uint64_t avail = ce - (b + have);                   // bits left in chunk k
        uint32_t take = 32 - have;
        if (take > avail) take = (uint32_t)avail;
        const uint32_t bitsv = (uint32_t)((pair << o) >> (64 - take));
        word |= bitsv << (32 - have - take);
        have += take;
        k++;
    }
    return word;
}

// One warp per chunk: the stream words whose last bit lies in the chunk, and
// the stream's partial final word in the last chunk.  Chunk c holds bits
// [cb, ce): it owns words [cb / 32, ce / 32), plus word total / 32 when it
// ends the stream on a partial word.
__global__ void __launch_bounds__(256) gather_kernel(const uint32_t *scratch, uint64_t slot, const uint64_t *offs,
                                                     uint64_t nchunks, uint32_t *out, uint64_t cap_words,
                                                     uint32_t *status) {
    const uint64_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31;
    if (c >= nchunks) return;
    const uint64_t cb = offs[c], ce = offs[c + 1], total = offs[nchunks];
    if (ce == cb) return;
    const uint64_t wf = cb / 32;
    uint64_t wl = ce / 32;
    if (ce == total && (total & 31)) wl = total / 32 + 1;
    bool over = false;
    for (uint64_t w = wf + lane; w < wl; w += 32) {
        // the word's first bit may lie in an earlier chunk (chunks hold >= 1 bit)
        const uint64_t b0 = 32 * w;
        uint64_t k = c;
        while (k > 0 && offs[k] > b0) k--;
        const uint32_t v = stream_word(scratch, slot, offs, nchunks, k, b0);
        if (w < cap_words) out[w] = v; else over = true;
    }
    if (over) set_error(status, HUFF_ERR_CAPACITY);
}

// Scratch of the three-kernel path for n symbols in chunks of 2^M: chunk
// lengths, then one slot per chunk of 2^(M-r) * Q words.
size_t shuffle_scratch_bytes(uint64_t n, int M, int r) {
    if (r < 0) r = 3;
    if (r > M) r = M;
    const uint64_t nchunks = (n + (1ull << M) - 1) >> M;
    const uint64_t Q = ((1ull << r) * kShufMaxLen + 31) / 32 + 1;
    return ((8 * nchunks + 255) & ~255ull) + nchunks * (1ull << (M - r)) * Q * 4 + 256;
}

template <typename Sym>
static huff_status launch_shuffle(const void *d_sym, uint64_t n, const void *d_codebook, uint32_t nbins,
                                  int M, int r, uint32_t max_len, uint32_t *d_out, uint64_t cap, uint64_t *d_offs,
                                  uint64_t *d_total, uint8_t *scratch, uint32_t *status, cudaStream_t st) {
    const uint64_t nchunks = (n + (1ull << M) - 1) >> M;
    if (r < 0) r = 3;                                         // the paper's choice (r is fixed at launch here)
    if (r > M) r = M;
    if (r > kShufMaxR || M - r > 10) return HUFF_ERR_INVALID_ARG;   // <= 16 symbols and <= 1024 threads
    (void)max_len;
    const uint32_t T = 1u << (M - r);
    const uint32_t Q = ((1u << r) * kShufMaxLen + 31) / 32 + 1;
    const uint64_t slot = (uint64_t)T * Q;
    uint64_t *chunk_bits = reinterpret_cast<uint64_t *>(scratch);
    uint32_t *data = reinterpret_cast<uint32_t *>(scratch + ((8 * nchunks + 255) & ~255ull));
    const size_t smem = (size_t)slot * 4;
    void (*kern)(ShufArgs) = shuffle_merge_kernel<Sym>;
    if (!allow_dynamic_smem((const void *)kern, smem)) return HUFF_ERR_INVALID_ARG;
    ShufArgs a;
    a.sym = static_cast<const uint8_t *>(d_sym);
    a.n = n;
    a.cw = reinterpret_cast<const uint64_t *>(static_cast<const uint8_t *>(d_codebook) + cb_cw_offset());
    a.nbins = nbins;
    a.M = M;
    a.r = r;
    a.slot_words = Q;
    a.scratch = data;
    a.chunk_bits = chunk_bits;
    a.status = status;
    kern<<<(unsigned)nchunks, T, smem, st>>>(a);
    chunk_scan_kernel<<<1, kScanThreads, 0, st>>>(chunk_bits, nchunks, d_offs, d_total);
    const uint64_t gthreads = nchunks * 32;
    gather_kernel<<<(unsigned)((gthreads + 255) / 256), 256, 0, st>>>(data, slot, d_offs, nchunks, d_out, cap,
                                                                      status);
    note_launch(3);
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

huff_status encode_shuffle_launch(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook,
                                  uint32_t nbins, int chunk_log2, int reduce_log2, uint32_t max_len, uint32_t *d_out,
                                  uint64_t cap, uint64_t *d_offs, uint64_t *d_total, uint8_t *scratch,
                                  uint32_t *status, cudaStream_t st) {
    switch (dtype) {
        case HUFF_U8: return launch_shuffle<uint8_t>(d_sym, n, d_codebook, nbins, chunk_log2, reduce_log2, max_len, d_out, cap, d_offs, d_total, scratch, status, st);
        case HUFF_U16: return launch_shuffle<uint16_t>(d_sym, n, d_codebook, nbins, chunk_log2, reduce_log2, max_len, d_out, cap, d_offs, d_total, scratch, status, st);
        case HUFF_U32: return launch_shuffle<uint32_t>(d_sym, n, d_codebook, nbins, chunk_log2, reduce_log2, max_len, d_out, cap, d_offs, d_total, scratch, status, st);
    }
    return HUFF_ERR_INVALID_ARG;
}

}  // namespace huff
