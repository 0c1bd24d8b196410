// Treeless canonical decoding (Sec. IV-B2): a codeword of length l is the
// first l-bit window v with v >= First[l]; its symbol is
// sorted_syms[Entry[l] + v - First[l]].  The chunk offsets written by the
// encoder let every chunk be decoded independently: one thread per chunk.
//
// GB300 form.  Every CTA first tabulates that rule in shared memory:
//   level 1, over windows of L = min(max_len, 12) bits: symbol << 10 | length
//     for a code of at most L bits, kDecInvalid when no code starts there, and
//     for a prefix of longer codes either kDecLong | subtable << 10 or 0;
//   level 2, one subtable of 2^(max_len - L) entries per such prefix, indexed
//     by the next max_len - L bits, when they fit (at most kL2Bits bits and
//     kL2Entries entries in all).
// So a code costs one or two shared lookups; prefixes left at 0 continue the
// First/Entry search from length L + 1 on the register buffer (First, Entry
// and Count in shared memory).  For alphabets of at most 1,024 symbols and
// fields of few chunks, a pair table over the same windows gives two codes
// per lookup when both fit in the window.  The stream
// is read through a 64-bit register buffer refilled 32 bits at a time, and
// decoded symbols are packed into 32-byte vector stores (one per
// 32 / sizeof(sym) symbols), since neighbouring lanes write 2^M symbols apart.
#include <type_traits>

#include "kernels.cuh"

namespace huff {

constexpr int kDecThreads = 256;
constexpr uint32_t kLutBits = 12;
constexpr uint32_t kDecPairBins = 1024;     // two-code table entries for alphabets up to this size
constexpr uint32_t kDecSymShift = 10;       // table entries: symbol (up to 22 bits) << kDecSymShift | length
constexpr uint32_t kDecInvalid = 0x200u;    // table entry: no codeword starts with this window
constexpr uint32_t kDecLong = 0x100u;       // level-1 entry: prefix of longer codes, subtable index from bit 10
constexpr uint32_t kL2Bits = 8;             // longest level-2 index
constexpr uint32_t kL2Entries = 4096;       // level-2 entries in all

// Per-CTA decoding tables (file scope so the out-of-line search reads them
// as shared memory).
__shared__ uint64_t dec_first[HUFF_MAX_LEN + 1];
__shared__ uint32_t dec_entry[HUFF_MAX_LEN + 1];
__shared__ uint32_t dec_count[HUFF_MAX_LEN + 1];
__shared__ uint32_t dec_lut[1u << kLutBits];
__shared__ uint32_t dec_lut2[kL2Entries];
__shared__ uint32_t dec_nlong[kDecThreads / 32 + 1];
__shared__ uint16_t dec_lpfx[kL2Entries / 2];   // level-1 window of each numbered long prefix
__shared__ uint32_t dec_pair[1u << kLutBits];

struct DecArgs {
    const uint32_t *in;   // whole 32-bit words of the stream's units
    uint64_t total_bits;
    uint64_t in_words;
    const uint64_t *offs;
    int chunk_log2;
    uint64_t n;
    uint64_t nchunks;
    const uint8_t *book;
    uint8_t *out;
    uint32_t nbins;
    int vec_out;          // out is 16-byte aligned and a chunk is a whole number of 16-byte runs
    int pair_out;         // out is 8-byte aligned and a chunk is a whole number of 8-byte runs
    uint32_t *status;
    uint32_t perm;        // byte order of a loaded word into stream order: identity for 32-bit
                          // units, halves swapped for 16-bit, bytes reversed for 8-bit
    uint32_t off_shift;   // chunk offsets count units of 2^off_shift bits (0: bits)
    uint32_t unit_mask;   // chunk-aligned layout: unit bits - 1 (a chunk ends within its last unit); 0: dense
};

__device__ __forceinline__ uint32_t ld_word(const uint32_t *in, uint64_t nwords, uint64_t w, uint32_t perm) {
    return w < nwords ? __byte_perm(__ldg(in + w), 0u, perm) : 0u;
}

// The stream's bits [p, p + 64), MSB first (zeros past the end).
__device__ __forceinline__ uint64_t window64(const uint32_t *in, uint64_t nwords, uint64_t p, uint32_t perm) {
    const uint64_t w = p >> 5;
    const uint32_t sh = p & 31;
    const uint64_t a = ld_word(in, nwords, w, perm), b = ld_word(in, nwords, w + 1, perm),
                   c = ld_word(in, nwords, w + 2, perm);
    const uint64_t hi = (a << 32) | b;
    return sh ? (hi << sh) | (c >> (32 - sh)) : hi;
}

// A code longer than the table: the First/Entry search from length L + 1 on
// the window `win` of the stream at the code's start (valid for max_len bits).
// Returns sym << 8 | len, or 0 when no codeword starts there.  Out of line:
// only long codes come here.
__device__ __noinline__ uint32_t decode_long(uint64_t win, uint32_t L, uint32_t max_len, const uint32_t *gsyms) {
    for (uint32_t l = L + 1; l <= max_len; l++) {
        const uint64_t v = win >> (64 - l);
        if (v >= dec_first[l]) {
            if (v - dec_first[l] >= dec_count[l]) return 0;
            return (__ldg(gsyms + dec_entry[l] + (uint32_t)(v - dec_first[l])) << 8) | l;
        }
    }
    return 0;
}

// One chunk: symbols [i0, i1) from stream bits [p0, pend).  Stops at the
// first invalid code; reports it, and a chunk that does not end exactly at
// pend, through the status word.  Reads are bounded by the stream and writes
// by the chunk, whatever the stream holds.
template <int W, bool FMT>
__device__ __forceinline__ void decode_chunk(const DecArgs &a, const uint32_t *gsyms, bool pair, uint32_t L,
                                             uint32_t max_len, uint64_t i0, uint64_t i1, uint64_t p0, uint64_t pend) {
    using Sym = typename std::conditional<W == 1, uint8_t, typename std::conditional<W == 2, uint16_t, uint32_t>::type>::type;
    Sym *out = reinterpret_cast<Sym *>(a.out);
    // Word indices are relative to the chunk's first word cw0 (32-bit: a chunk
    // spans far fewer than 2^32 words; lim stops reads at the stream's end).
    // The buffer (hi:lo) holds the stream's bits [p, p + nb) MSB first; nxt
    // holds the word that follows them, already loaded, and wn is the word after
    // nxt, so p = 32 * (cw0 + wn - 1) - nb at all times.  A refill splices nxt
    // in and starts loading the next word, which is not needed before the next
    // refill: the load's latency hides behind the symbols in between.
    const uint64_t cw0 = p0 >> 5;
    const uint32_t *cin = a.in + cw0;
    const uint64_t left = a.in_words > cw0 ? a.in_words - cw0 : 0;
    const uint32_t lim = left < 0xFFFFFFFFull ? (uint32_t)left : 0xFFFFFFFFu;
    // FMT: a stream of 8- or 16-bit units or the chunk-aligned layout (words
    // permuted into stream order, offsets in units, padded chunk ends)
    const uint32_t perm = FMT ? a.perm : 0x3210u;
    auto word = [&](uint32_t k) {
        const uint32_t w = k < lim ? __ldg(cin + k) : 0u;
        return FMT ? __byte_perm(w, 0u, perm) : w;
    };
    uint32_t hi, lo, nb, wn, nxt;
    auto start = [&](uint64_t p) {
        wn = (uint32_t)((p >> 5) - cw0);
        const uint32_t sh = p & 31, w0 = word(wn), w1 = word(wn + 1);
        nxt = word(wn + 2);
        hi = __funnelshift_l(w1, w0, sh);
        lo = w1 << sh;
        nb = 64 - sh;
        wn += 3;
    };
    auto pos = [&]() { return 32 * (cw0 + wn - 1) - nb; };
    start(p0);
    const uint32_t shL = 32 - L;
    // level-2 index: stream bits L..max_len-1 (used only when max_len - L <= kL2Bits)
    const uint32_t sh2 = 32 - (max_len <= 32 ? max_len : 32), m2 = max_len - L <= kL2Bits ? (1u << (max_len - L)) - 1 : 0u;
    bool ok = true;
    // refill: nxt goes to buffer bits [nb, nb + 32), then the following word
    // is loaded into nxt (predicated, no branch)
    auto refill = [&]() {
        const bool need = nb <= 32;
        const uint32_t w = need ? nxt : 0u;
        hi |= __funnelshift_rc(w, 0u, nb);
        lo |= __funnelshift_lc(0u, w, 32 - nb);
        if (need) nxt = word(wn);
        wn += need;
        nb += need ? 32u : 0u;
    };
    // one code from a refilled buffer
    auto single = [&](uint32_t &s) {
        uint32_t e = dec_lut[hi >> shL];
        if (e & kDecLong) e = dec_lut2[(e >> kDecSymShift) * (m2 + 1) + ((hi >> sh2) & m2)];
        uint32_t l = e & 0xFFu;
        s = e >> kDecSymShift;
        if (l == 0) {
            // no code (kDecInvalid), or longer than the tables: the search, on
            // the buffer when it holds max_len bits, else on a fresh window
            uint32_t r = 0;
            if (e == 0) {
                const uint64_t win = max_len <= nb ? ((uint64_t)hi << 32 | lo) : window64(a.in, a.in_words, pos(), perm);
                r = decode_long(win, L, max_len, gsyms);
            }
            if (r == 0) { ok = false; return; }
            s = r >> 8;
            l = r & 0xFFu;
            if (l > nb) { start(pos() + l); return; }
            if (l >= 32) {
                hi = l < 64 ? lo << (l - 32) : 0u;
                lo = 0;
                nb -= l;
                return;
            }
        }
        // consume l (1..31) bits
        hi = __funnelshift_l(lo, hi, l);
        lo <<= l;
        nb -= l;
    };
    auto next = [&](uint32_t &s) {
        refill();
        single(s);
    };
    uint64_t i = i0;
    bool paired = false;
    if constexpr (W <= 2) {
    if (pair) {
        paired = true;
        // Two codes per lookup where a 12-bit window holds both (the pair table);
        // symbols gather in a 64-bit register of 8 / W slots, written 8 bytes at
        // a time (the chunk and the output are 8-byte aligned here).
        constexpr uint32_t kSlots = 8 / W, kSymBits = 8 * W, kSymMask = W == 1 ? 0xFFu : 0xFFFFu;
        uint64_t obuf = 0;
        uint32_t oc = 0;
        auto put = [&](uint32_t s) {
            obuf |= (uint64_t)s << (kSymBits * oc);
            if (++oc == kSlots) {
                *reinterpret_cast<uint64_t *>(out + i) = obuf;
                i += kSlots;
                obuf = 0;
                oc = 0;
            }
        };
        while (i + oc < i1 && ok) {
            refill();
            const uint32_t e2 = dec_pair[hi >> shL];
            uint32_t l1 = (e2 >> 20) & 15u;
            if (l1 != 0) {
                // take the second code only while the chunk still needs a symbol
                const uint32_t l2 = i + oc + 1 < i1 ? (e2 >> 24) & 15u : 0u;
                const uint32_t l = l1 + l2;          // at most 12
                hi = __funnelshift_l(lo, hi, l);
                lo <<= l;
                nb -= l;
                put(e2 & 0x3FFu);
                if (l2) put((e2 >> 10) & 0x3FFu);
            } else {
                uint32_t sym = 0;
                single(sym);
                if (ok) put(sym);
            }
        }
        // the last partial group
        for (uint32_t k = 0; k < oc && ok; k++) out[i + k] = (Sym)((obuf >> (kSymBits * k)) & kSymMask);
        if (ok) i += oc;
    }
    }
    if (!paired && a.vec_out) {
        constexpr int kBatch = 32 / W;          // symbols per 32-byte store
        for (; i + kBatch <= i1 && ok; i += kBatch) {
            uint32_t r[8];
#pragma unroll
            for (int k = 0; k < kBatch; k++) {
                uint32_t s = 0;
                next(s);
                constexpr int kPer = 4 / W;
                constexpr uint32_t kMask = W == 4 ? 0xFFFFFFFFu : (1u << (8 * (W & 3))) - 1;
                const int slot = k / kPer, shift = (k % kPer) * 8 * W;
                r[slot] = (k % kPer == 0) ? (s & kMask) : r[slot] | ((s & kMask) << shift);
            }
            if (!ok) break;
            uint4 *dst = reinterpret_cast<uint4 *>(out + i);
            dst[0] = make_uint4(r[0], r[1], r[2], r[3]);
            dst[1] = make_uint4(r[4], r[5], r[6], r[7]);
        }
    }
    for (; i < i1 && ok; i++) {
        uint32_t s = 0;
        next(s);
        if (ok) out[i] = (Sym)s;
    }
    // dense: the chunk ends exactly at the next offset; chunk-aligned: within
    // the unit before it (the rest of that unit is padding)
    const uint64_t pe = pos();
    const uint64_t um = FMT ? a.unit_mask : 0u;
    if (!ok || pe > pend || ((pe + um) & ~um) != pend)
        set_error(a.status, HUFF_ERR_INVALID_ARG);
}

template <int W, bool FMT>
__global__ void __launch_bounds__(kDecThreads) decode_kernel(DecArgs a) {
    const huff_codebook_header *hdr = reinterpret_cast<const huff_codebook_header *>(a.book);
    const uint32_t *sorted_syms = reinterpret_cast<const uint32_t *>(a.book + cb_sorted_offset(a.nbins));
    const uint32_t max_len = hdr->max_len;
    if (hdr->nbins != a.nbins || max_len == 0 || max_len > HUFF_MAX_LEN) {
        if (threadIdx.x == 0) set_error(a.status, HUFF_ERR_INVALID_ARG);
        return;      // uniform over the CTA: every thread read the same header
    }
    for (int l = threadIdx.x; l <= HUFF_MAX_LEN; l += blockDim.x) {
        dec_first[l] = hdr->first[l];
        dec_entry[l] = hdr->entry[l];
        dec_count[l] = hdr->count[l];
    }
    __syncthreads();
    // level 1 over L-bit windows: the decoding rule restricted to lengths <= L;
    // each thread takes 2^L / kDecThreads consecutive windows (at least one)
    const uint32_t L = max_len < kLutBits ? max_len : kLutBits;
    const uint32_t nwin = 1u << L;
    const uint32_t per = nwin >= kDecThreads ? nwin / kDecThreads : 1;
    const uint32_t x0 = threadIdx.x * per;
    const uint32_t l2bits = max_len - L;
    uint32_t mylong = 0;
    for (uint32_t x = x0; x < x0 + per && x < nwin; x++) {
        uint32_t e = 0;       // a prefix of longer codes unless a length <= L decides
        for (uint32_t l = 1; l <= L; l++) {
            const uint64_t v = x >> (L - l);
            if (v >= dec_first[l]) {
                if (v - dec_first[l] < dec_count[l]) {
                    const uint32_t k = dec_entry[l] + (uint32_t)(v - dec_first[l]);
                    e = (__ldg(sorted_syms + k) << kDecSymShift) | l;
                } else {
                    e = kDecInvalid;
                }
                break;
            }
        }
        mylong += e == 0;
        dec_lut[x] = e;
    }
    // number the long prefixes in window order (a block scan of the counts)
    uint32_t inc = mylong;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if ((threadIdx.x & 31) >= o) inc += y;
    }
    if ((threadIdx.x & 31) == 31) dec_nlong[threadIdx.x >> 5] = inc;
    __syncthreads();
    uint32_t base = 0, total = 0;
    for (uint32_t w = 0; w < kDecThreads / 32; w++) {
        if (w < (threadIdx.x >> 5)) base += dec_nlong[w];
        total += dec_nlong[w];
    }
    base += inc - mylong;
    const bool two_level = l2bits >= 1 && l2bits <= kL2Bits && (total << l2bits) <= kL2Entries;
    if (two_level) {
        // total << l2bits <= kL2Entries with l2bits >= 1: every number fits dec_lpfx
        for (uint32_t x = x0; x < x0 + per && x < nwin; x++)
            if (dec_lut[x] == 0) {
                dec_lpfx[base] = (uint16_t)x;
                dec_lut[x] = kDecLong | (base++ << kDecSymShift);
            }
    }
    __syncthreads();
    if (two_level) {
        // level 2: entry (j, y) decodes the max_len-bit window (prefix_j << l2bits | y)
        for (uint32_t q = threadIdx.x; q < (total << l2bits); q += kDecThreads) {
            const uint32_t j = q >> l2bits, y = q & ((1u << l2bits) - 1);
            const uint64_t win = ((uint64_t)dec_lpfx[j] << l2bits) | y;     // max_len bits
            uint32_t e = kDecInvalid;
            for (uint32_t l = L + 1; l <= max_len; l++) {
                const uint64_t v = win >> (max_len - l);
                if (v >= dec_first[l]) {
                    if (v - dec_first[l] < dec_count[l]) {
                        const uint32_t k = dec_entry[l] + (uint32_t)(v - dec_first[l]);
                        e = (__ldg(sorted_syms + k) << kDecSymShift) | l;
                    }
                    break;
                }
            }
            dec_lut2[q] = e;
        }
        __syncthreads();
    }
    // pair table over the same windows: s1 | s2 << 10 | len1 << 20 | len2 << 24
    // when the window holds a first code of at most L bits (len2 = 0 when no
    // second code fits in the rest of the window), 0 otherwise
    const bool pair = a.nbins <= kDecPairBins && a.pair_out && W <= 2;
    if (pair) {
        for (uint32_t x = threadIdx.x; x < nwin; x += kDecThreads) {
            const uint32_t e1 = dec_lut[x];
            const uint32_t l1 = e1 & 0xFFu;
            uint32_t e = 0;
            if (l1 != 0) {
                e = (e1 >> kDecSymShift) | (l1 << 20);
                // the rest of the window, shifted up; its low l1 bits are unknown,
                // so a second code counts only if it lies within the known bits
                const uint32_t x2 = (x << l1) & (nwin - 1);
                const uint32_t f = dec_lut[x2];
                const uint32_t l2 = f & 0xFFu;
                if (l2 != 0 && l2 <= L - l1) e |= ((f >> kDecSymShift) << 10) | (l2 << 24);
            }
            dec_pair[x] = e;
        }
        __syncthreads();
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < a.nchunks; c += stride) {
        const uint64_t i0 = c << a.chunk_log2;
        const uint64_t i1 = i0 + (1ull << a.chunk_log2) < a.n ? i0 + (1ull << a.chunk_log2) : a.n;
        const uint32_t osh = FMT ? a.off_shift : 0u;
        decode_chunk<W, FMT>(a, sorted_syms, pair, L, max_len, i0, i1, a.offs[c] << osh, a.offs[c + 1] << osh);
    }
}

huff_status decode_launch(const void *d_in, uint64_t total_bits, const uint64_t *d_offs, int chunk_log2,
                          uint32_t format, uint64_t n, huff_dtype dtype, const void *d_codebook, uint32_t nbins,
                          void *d_out, uint32_t *status, cudaStream_t st) {
    DecArgs a;
    a.in = static_cast<const uint32_t *>(d_in);
    a.total_bits = total_bits;
    a.in_words = (total_bits + 31) / 32;
    const uint32_t wlog = fmt_wlog(format);
    a.perm = wlog == 5 ? 0x3210u : wlog == 4 ? 0x1032u : 0x0123u;
    a.off_shift = fmt_chunk_aligned(format) ? wlog : 0u;
    a.unit_mask = fmt_chunk_aligned(format) ? (1u << wlog) - 1 : 0u;
    a.offs = d_offs;
    a.chunk_log2 = chunk_log2;
    a.n = n;
    a.nchunks = (n + (1ull << chunk_log2) - 1) >> chunk_log2;
    a.book = static_cast<const uint8_t *>(d_codebook);
    a.out = static_cast<uint8_t *>(d_out);
    a.nbins = nbins;
    // 32-byte stores need a 16-byte aligned output and chunks of whole 16-byte runs
    a.vec_out = ((uintptr_t)d_out & 15) == 0 && ((1ull << chunk_log2) * (uint64_t)dtype) % 16 == 0;
    // Two codes per lookup shorten each thread's serial chain, which is what
    // bounds a field of few chunks (at most one CTA of chunks per SM); with
    // more chunks the decode is issue-bound, and the one-code path's fixed
    // 32-byte batches (no divergence, whole sectors) are faster.
    a.pair_out = ((uintptr_t)d_out & 7) == 0 && ((1ull << chunk_log2) * (uint64_t)dtype) % 8 == 0 &&
                 a.nchunks <= (uint64_t)sm_count() * kDecThreads;
    a.status = status;
    if (a.nchunks == 0) return HUFF_OK;
    void (*kern)(DecArgs);
    if (format == 0)
        kern = dtype == HUFF_U8 ? decode_kernel<1, false> : dtype == HUFF_U16 ? decode_kernel<2, false> : decode_kernel<4, false>;
    else
        kern = dtype == HUFF_U8 ? decode_kernel<1, true> : dtype == HUFF_U16 ? decode_kernel<2, true> : decode_kernel<4, true>;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kDecThreads, 0);
    if (occ < 1) occ = 1;
    uint64_t grid = (a.nchunks + kDecThreads - 1) / kDecThreads;
    const uint64_t resident = (uint64_t)sm_count() * occ;
    if (grid > resident) grid = resident;
    kern<<<(unsigned)grid, kDecThreads, 0, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

}  // namespace huff
