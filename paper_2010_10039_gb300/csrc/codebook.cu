// Codebook construction (Sec. IV-B, Algorithm 1) in one CTA.
//
// GenerateCL.  The paper runs the parallel construction of Ostadzadeh et al.:
// every round makes t from the two lightest nodes, selects the leaves lighter
// than t, merges them with the waiting joined nodes (Merge Path) and melds
// adjacent pairs.  Here one round does the same with a tie rule that makes the
// result identical to the serial two-queue construction (leaves ordered by
// (count, id), a leaf before a joined node of equal weight, joined nodes in
// creation order):
//   S      = the waiting leaves and joined nodes in that order (a stable
//            leaf-first merge of two sorted queues),
//   t      = weight(S0) + weight(S1),
//   k      = number of nodes in S of weight <= t,
//   m      = k rounded down to even,
//   meld S[2j] with S[2j+1] for j < m/2, appending the results in order j.
// Every node of weight <= t leaves the queues before the node S0+S1 in the
// serial order (equal-weight leaves win the tie, equal-weight joined nodes
// are older), and the pairs leave two by two, so the serial construction melds
// exactly these pairs; an odd k leaves S[k-1] to pair with S0+S1 next round.
// The paper's sync-separated parallel regions become one 1024-thread CTA with
// a single barrier per round: every warp derives the round's t and node counts
// itself (the same reads give the same result), and thread j melds pair j
// after finding S[2j] by a Merge Path co-ranking search in the two queues, so
// the merged order is never materialised.
//
// Lengths.  Instead of walking every leaf to its leader each round
// (UpdateLeafNode), each meld records the parent of its two inputs; after the
// last round a leaf's length is the number of parent links from it to the root.
//
// GenerateCW + canonisation (Sec. IV-B2).  Code lengths are counted per
// length; First is filled from the longest length down so that a shorter
// codeword is numerically larger than the prefixes of longer ones; codewords of
// one length are consecutive in ascending symbol id (a warp-match rank inside
// each 1024-id slice plus a per-length running base).  Entry and the
// (length, id)-sorted symbol list form the reverse codebook.
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace huff {

constexpr int kCbThreads = 1024;
constexpr uint32_t kCbSmemBins = 4096;     // arrays live in shared memory up to this alphabet
constexpr uint32_t kCbRevDepth = 16384;    // above this many used symbols, depths by a per-round pass
constexpr uint32_t kRadixDigits = 256;     // 8-bit digits of the large-alphabet sort
constexpr uint32_t kRhStride = 34;         // u16 per digit row of the counting table: 17 words, odd, so
                                           // one warp's distinct digits fall in distinct banks
constexpr uint32_t kSmallAlphabet = 65536; // above this the sort keys carry 32-bit ids and the
                                           // counting table 32-bit slots (BIG instantiations)

// Counting-table slot type and row stride (odd in words) of the two forms.
template <bool BIG> struct RhOf { using T = uint16_t; static constexpr uint32_t kStride = kRhStride; };
template <> struct RhOf<true> { using T = uint32_t; static constexpr uint32_t kStride = 33; };

struct CbArrays {
    uint64_t *keys;     // 2P      sort keys (count << 16 | id); the two halves are the
                        //         exchange buffers of the sorts
    uint32_t *wL;       // m       leaf weights (sorted)
    uint32_t *wI;       // m       joined-node weights (creation order)
    uint32_t *parent;   // 2m      parent node id of every node (leaves 0..m-1, joined m..2m-2)
    uint32_t *rstart;   // m       first joined node of each round     } alphabets above
    uint32_t *depthI;   // m       depth of each joined node           } kCbSmemBins only
    uint8_t *lenS;      // nbins   length by symbol id
};

__host__ __device__ inline uint32_t pow2_ceil(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t cb_array_bytes(uint32_t nbins) {
    size_t P = pow2_ceil(nbins);
    const size_t rev = nbins > kCbSmemBins ? 2 * align16((size_t)nbins * 4) : 0;
    return align16(P * 16) + 2 * align16((size_t)nbins * 4) + align16((size_t)nbins * 8) + rev + align16(nbins);
}

__device__ inline CbArrays cb_carve(uint8_t *p, uint32_t nbins) {
    CbArrays a;
    size_t P = pow2_ceil(nbins);
    a.keys = reinterpret_cast<uint64_t *>(p); p += align16(P * 16);
    a.wL = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 4);
    a.wI = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 4);
    a.parent = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 8);
    a.rstart = a.depthI = nullptr;
    if (nbins > kCbSmemBins) {
        a.rstart = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 4);
        a.depthI = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 4);
    }
    a.lenS = p;
    return a;
}

// Bitonic stages of stride j < 32 for the keys this thread holds (element
// e = tid + r * kCbThreads; the partner e ^ j is in the same warp, so the
// exchange is a shuffle, not a barrier-separated pass).
__device__ __forceinline__ uint64_t bitonic_warp_stages(uint64_t x, uint32_t e, uint32_t k, uint32_t jmax) {
    for (uint32_t j = jmax; j > 0; j >>= 1) {
        const uint64_t y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
        const bool up = (e & k) == 0, lower = (e & j) == 0;
        x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
    }
    return x;
}

// Ascending bitonic sort of P <= kCbThreads keys, thread e holding element e
// (threads e >= P hold ~0 and are never read).  Strides of 32 and more go
// through shared memory, alternating between buf[0, P) and buf[P, 2P) so that
// one barrier per stride suffices; smaller strides are shuffles.
__device__ __forceinline__ uint64_t bitonic_sort_regs(uint64_t x, uint32_t P, uint64_t *buf) {
    const uint32_t e = threadIdx.x;
    uint32_t flip = 0;
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j >= 32; j >>= 1) {
            uint64_t *b = buf + flip * P;
            flip ^= 1;
            if (e < P) b[e] = x;
            __syncthreads();
            if (e < P) {
                const uint64_t y = b[e ^ j];
                const bool up = (e & k) == 0, lower = (e & j) == 0;
                x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
            }
        }
        // within a warp: lanes below P pair only with lanes below P
        x = bitonic_warp_stages(x, e, k, (k >> 1) < 16 ? (k >> 1) : 16);
    }
    return x;
}

// ---- stable counting passes (one CTA)
// A pass places elements 0..len-1 that carry a digit (0..kRadixDigits-1) in
// digit-major, then element order.  Warp w owns a contiguous segment of the
// elements; its per-digit counts rh[digit][w], scanned in digit-major order,
// give its first slot for each digit, and the lanes of one step rank among
// themselves by a warp match.  Up to 65,536 elements the counts and slots stay
// below 65,536 and the table is u16, its rows padded to kRhStride; larger
// alphabets (BIG) take u32 slots.
// elem(i) returns an element, four at a time so that their loads overlap.

struct CpElem {
    bool valid;         // carries a digit
    uint32_t digit;
    uint64_t payload;
};

__device__ __forceinline__ void cp_segment(uint32_t len, uint32_t &begin, uint32_t &end) {
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t seg = (((len + 31) / 32) + 31) & ~31u;
    begin = warp * seg < len ? warp * seg : len;
    end = begin + seg < len ? begin + seg : len;
}

// Counts, then scans rh into first slots; totals[d] (d < ntotals) receives the
// number of elements with digit d.  Ends with a barrier.  Counting needs no
// ranks: ATOMIC counts with one shared atomic per element (on the 32-bit word
// holding rh[digit][warp]; a count stays below 65,536, so nothing carries
// into the neighbour), which beats the warp match when a step holds many
// distinct digits; the match wins when they repeat.
template <bool ATOMIC, typename Elem, typename Slot, uint32_t STRIDE>
__device__ void cpass_count(uint32_t len, Elem elem, Slot (*rh)[STRIDE], uint32_t *wsum, uint32_t *totals,
                            uint32_t ntotals) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1;
    uint32_t begin, end;
    cp_segment(len, begin, end);
    for (uint32_t i = tid; i < kRadixDigits * STRIDE; i += kCbThreads) (&rh[0][0])[i] = 0;
    __syncthreads();
    for (uint32_t b = begin; b < end; b += 128) {
        CpElem e[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = b + 32 * q + lane;
            e[q] = i < end ? elem(i) : CpElem{false, 0u, 0ull};
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (ATOMIC) {
                if (e[q].valid) {
                    if (sizeof(Slot) == 2)
                        atomicAdd(reinterpret_cast<uint32_t *>(&rh[e[q].digit][warp & ~1u]), 1u << (16 * (warp & 1)));
                    else
                        atomicAdd(reinterpret_cast<uint32_t *>(&rh[e[q].digit][warp]), 1u);
                }
            } else {
                const uint32_t peers = __match_any_sync(0xFFFFFFFFu, e[q].valid ? e[q].digit : 0x10000u);
                if (e[q].valid && __popc(peers & lt) == 0) rh[e[q].digit][warp] += (Slot)__popc(peers);
            }
        }
    }
    __syncthreads();
    for (uint32_t d = tid; d < ntotals; d += kCbThreads) {
        uint32_t t = 0;
        for (uint32_t w = 0; w < 32; w++) t += rh[d][w];
        totals[d] = t;
    }
    // exclusive scan in digit-major order: eight entries per thread (digit
    // tid / 4, warps 8 * (tid % 4) ..)
    Slot *row = &rh[tid >> 2][8 * (tid & 3)];
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) { v[q] = row[q]; sum += v[q]; }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t wbase = 0;
    for (uint32_t w = 0; w < warp; w++) wbase += wsum[w];
    uint32_t run = wbase + inc - sum;
#pragma unroll
    for (int q = 0; q < 8; q++) { row[q] = (Slot)run; run += v[q]; }
    __syncthreads();
}

// Hands every element with a digit to place(slot, payload) and every other
// one to skip(payload), in the same element order as cpass_count.  Ends with
// a barrier.
template <typename Elem, typename Place, typename Skip, typename Slot, uint32_t STRIDE>
__device__ void cpass_scatter(uint32_t len, Elem elem, Place place, Skip skip, Slot (*rh)[STRIDE]) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1;
    uint32_t begin, end;
    cp_segment(len, begin, end);
    for (uint32_t b = begin; b < end; b += 128) {
        CpElem e[4];
        bool in[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = b + 32 * q + lane;
            in[q] = i < end;
            e[q] = in[q] ? elem(i) : CpElem{false, 0u, 0ull};
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, e[q].valid ? e[q].digit : 0x10000u);
            const uint32_t rank = __popc(peers & lt);
            const uint32_t slot = e[q].valid ? rh[e[q].digit][warp] : 0u;
            __syncwarp();
            if (e[q].valid && rank == 0) rh[e[q].digit][warp] = (Slot)(slot + __popc(peers));
            __syncwarp();
            if (e[q].valid) place(slot + rank, e[q].payload);
            else if (in[q]) skip(e[q].payload);
        }
    }
    __syncthreads();
}

// Stable LSD radix sort, by count, of the used bins of hist[nbins] into
// buf[0, m) as keys count << IDB | id (IDB = 16, or 32 above 65,536 bins).  Bins enter in id order, so equal counts
// stay in id order and the result is the (count, id) order.  8-bit digits,
// as many passes as maxcount has digits; pass 0 reads the histogram and drops
// unused bins, and the passes alternate between buf[0, P) and buf[P, 2P) so
// that the last one lands in buf[0, P).
template <bool BIG>
__device__ void radix_sort_keys(const uint32_t *hist, uint32_t nbins, uint32_t m, uint32_t maxcount, uint64_t *buf,
                                uint32_t P, typename RhOf<BIG>::T (*rh)[RhOf<BIG>::kStride], uint32_t *wsum) {
    constexpr uint32_t IDB = BIG ? 32 : 16;
    const uint32_t bits = 32 - __clz(maxcount);
    const uint32_t npass = bits > 8 ? (bits + 7) / 8 : 1;
    for (uint32_t pass = 0; pass < npass; pass++) {
        const uint32_t shift = IDB + 8 * pass;
        const uint64_t *src = buf + ((npass - pass) & 1) * P;
        uint64_t *dst = buf + ((npass - 1 - pass) & 1) * P;
        auto elem = [&](uint32_t i) -> CpElem {
            uint64_t key;
            if (pass == 0) {
                const uint32_t c = hist[i];
                key = ((uint64_t)c << IDB) | i;
                if (c == 0) return CpElem{false, 0u, key};
            } else {
                key = src[i];
            }
            return CpElem{true, (uint32_t)(key >> shift) & (kRadixDigits - 1), key};
        };
        const uint32_t len = pass == 0 ? nbins : m;
        // the low byte of varied counts spreads over many digits per step
        if (pass == 0 && maxcount >= 256) cpass_count<true>(len, elem, rh, wsum, nullptr, 0);
        else cpass_count<false>(len, elem, rh, wsum, nullptr, 0);
        cpass_scatter(len, elem, [&](uint32_t slot, uint64_t key) { dst[slot] = key; }, [](uint64_t) {}, rh);
    }
}

// Upper bounds of t in the sorted ranges wa[alo, ahi) and wb[blo, bhi) (index
// of the first element > t), one warp searching both side by side so that
// their loads overlap.
__device__ __forceinline__ void warp_upper_bound2(const uint32_t *wa, uint32_t alo, uint32_t ahi,
                                                  const uint32_t *wb, uint32_t blo, uint32_t bhi, uint32_t t,
                                                  uint32_t &ra, uint32_t &rb) {
    const uint32_t lane = threadIdx.x & 31;
    bool adone = false, bdone = false;
    while (true) {
        const bool awide = !adone && ahi - alo > 32, bwide = !bdone && bhi - blo > 32;
        if (!awide && !bwide) break;
        const uint32_t as = (ahi - alo + 31) / 32, bs = (bhi - blo + 31) / 32;
        const uint32_t ap = alo + lane * as, bp = blo + lane * bs;
        const bool pa = awide && ap < ahi && wa[ap] <= t;
        const bool pb = bwide && bp < bhi && wb[bp] <= t;
        const uint32_t ca = __popc(__ballot_sync(0xFFFFFFFFu, pa));
        const uint32_t cb = __popc(__ballot_sync(0xFFFFFFFFu, pb));
        if (awide) {
            if (ca == 0) { ahi = alo; adone = true; }
            else { const uint32_t nhi = alo + ca * as; alo = alo + (ca - 1) * as + 1; ahi = nhi < ahi ? nhi : ahi; }
        }
        if (bwide) {
            if (cb == 0) { bhi = blo; bdone = true; }
            else { const uint32_t nhi = blo + cb * bs; blo = blo + (cb - 1) * bs + 1; bhi = nhi < bhi ? nhi : bhi; }
        }
    }
    const bool pa = alo + lane < ahi && wa[alo + lane] <= t;
    const bool pb = blo + lane < bhi && wb[blo + lane] <= t;
    ra = alo + __popc(__ballot_sync(0xFFFFFFFFu, pa));
    rb = blo + __popc(__ballot_sync(0xFFFFFFFFu, pb));
}

// index of the first element > t in sorted w[lo, hi), one warp cooperating
__device__ uint32_t warp_upper_bound(const uint32_t *w, uint32_t lo, uint32_t hi, uint32_t t) {
    const uint32_t lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        uint32_t step = (hi - lo + 31) / 32;
        uint32_t pos = lo + lane * step;
        bool pred = pos < hi && w[pos] <= t;
        uint32_t cnt = __popc(__ballot_sync(0xFFFFFFFFu, pred));
        if (cnt == 0) return lo;
        uint32_t nlo = lo + (cnt - 1) * step + 1;
        uint32_t nhi = lo + cnt * step;
        if (nhi > hi) nhi = hi;
        lo = nlo;
        hi = nhi;
    }
    bool pred = lo + lane < hi && w[lo + lane] <= t;
    return lo + __popc(__ballot_sync(0xFFFFFFFFu, pred));
}

// Builds the codebook of one histogram with the whole CTA; `arrays` holds the
// construction's arrays (shared memory for small alphabets).  BIG: alphabets
// above 65,536 bins (32-bit ids in the sort keys, 32-bit counting slots).
template <bool BIG>
__device__ __forceinline__ void codebook_body(const CbArgs &g, uint8_t *arrays) {
    constexpr uint32_t IDB = BIG ? 32 : 16;
    constexpr uint64_t kIdMask = (1ull << IDB) - 1;
    __shared__ uint64_t s_sum, s_tbits;
    __shared__ uint32_t s_m, s_maxlen, s_bad, s_maxc, s_rounds;
    __shared__ uint32_t s_wsum[kCbThreads / 32];
    __shared__ typename RhOf<BIG>::T s_rh[kRadixDigits][RhOf<BIG>::kStride];
    __shared__ uint32_t s_count[HUFF_MAX_LEN + 1];
    __shared__ uint32_t s_base[HUFF_MAX_LEN + 1];
    __shared__ uint64_t s_first[HUFF_MAX_LEN + 1];
    __shared__ uint32_t s_entry[HUFF_MAX_LEN + 1];
    __shared__ uint32_t s_wcnt[kCbThreads / 32][HUFF_MAX_LEN + 1];

    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nbins = g.nbins;
    const uint32_t P = pow2_ceil(nbins);
    const bool small = P <= kCbThreads;      // one bin per thread: keys stay in registers
    CbArrays A = cb_carve(arrays, nbins);
    huff_codebook_header *hdr = reinterpret_cast<huff_codebook_header *>(g.book);
    uint64_t *cw = reinterpret_cast<uint64_t *>(g.book + cb_cw_offset());
    uint32_t *sorted_syms = reinterpret_cast<uint32_t *>(g.book + cb_sorted_offset(nbins));

    if (tid == 0) { s_sum = 0; s_tbits = 0; s_m = 0; s_bad = 0; s_maxlen = 0; s_maxc = 0; s_rounds = 0; }
    if (tid <= HUFF_MAX_LEN) { s_count[tid] = 0; s_base[tid] = 0; s_first[tid] = 0; s_entry[tid] = 0; }
    for (uint32_t i = tid; i < (kCbThreads / 32) * (HUFF_MAX_LEN + 1); i += kCbThreads) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();

    // ---- keys (one per thread up to kCbThreads bins), used count, largest
    // count, histogram sum
    uint64_t part = 0, mykey = ~0ull;
    uint32_t used = 0, mycount = 0, maxc = 0;
    for (uint32_t i = tid; i < nbins; i += kCbThreads) {
        const uint32_t c = g.hist[i];
        part += c;
        used += c != 0;
        maxc = c > maxc ? c : maxc;
        A.lenS[i] = 0;
        mycount = c;
        if (small && c) mykey = ((uint64_t)c << IDB) | i;
    }
    for (int o = 16; o; o >>= 1) {
        part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        used += __shfl_xor_sync(0xFFFFFFFFu, used, o);
        maxc = max(maxc, __shfl_xor_sync(0xFFFFFFFFu, maxc, o));
    }
    if (lane == 0) {
        atomicAdd((unsigned long long *)&s_sum, (unsigned long long)part);
        atomicAdd(&s_m, used);
        atomicMax(&s_maxc, maxc);
    }
    __syncthreads();
    const bool overflow = s_sum >= (1ull << 32);
    const uint32_t m = overflow ? 0 : s_m;
    if (overflow && tid == 0) set_error(g.status, HUFF_ERR_HIST_OVERFLOW);

    if (m >= 2) {
        // ---- bitonic sort of the keys (ascending: count, then id; unused last)
        if (small) {
            // Sparse histograms: compact the used keys to threads 0..m-1 first
            // (ranks by ballot), so only pow2_ceil(m) keys are sorted.
            uint32_t Ps = P;
            if (pow2_ceil(m) < P) {
                Ps = pow2_ceil(m);
                const bool u = mykey != ~0ull;
                const uint32_t bal = __ballot_sync(0xFFFFFFFFu, u);
                if (lane == 0) s_wsum[warp] = __popc(bal);
                __syncthreads();
                uint32_t r = __popc(bal & ((1u << lane) - 1));
                for (uint32_t w = 0; w < warp; w++) r += s_wsum[w];
                if (u) A.keys[r] = mykey;
                __syncthreads();
                mykey = tid < m ? A.keys[tid] : ~0ull;
            }
            // the exchange buffers are keys[0, 2Ps): every thread must be done
            // reading them before the sorted keys go back to keys[0, Ps)
            mykey = bitonic_sort_regs(mykey, Ps, A.keys);
            __syncthreads();
            if (tid < Ps) A.keys[tid] = mykey;
        } else {
            radix_sort_keys<BIG>(g.hist, nbins, m, s_maxc, A.keys, P, s_rh, s_wsum);
        }
        __syncthreads();
        for (uint32_t i = tid; i < m; i += kCbThreads) A.wL[i] = (uint32_t)(A.keys[i] >> IDB);
        __syncthreads();

        // ---- GenerateCL rounds.  c leaves and the joined nodes before ih have
        // been melded; joined nodes ih..it-1 wait.  The first rt threads run the
        // rounds (every warp repeats the selection, so fewer warps repeat less
        // of it; larger alphabets have more pairs per round and get more) and
        // all track the same (c, ih, it).  Within a round the reads (wL,
        // wI[ih, it)) and the writes (wI[it, it + pairs), parent) never
        // overlap, so one named barrier per round suffices.
        const uint32_t rt = m <= 2048 ? 256u : (m <= 16384 ? 512u : (uint32_t)kCbThreads);
        const bool rev = m > kCbRevDepth;      // implies nbins > kCbSmemBins: rstart exists
        if (tid < rt) {
            constexpr uint64_t kNone = 1ull << 33;     // above every weight (totals are < 2^32)
            uint32_t c = 0, ih = 0, it = 0, round = 0;
            while ((m - c) + (it - ih) >= 2) {
                if (rev && tid == 0) A.rstart[round] = it;
                round++;
                // t: the two lightest nodes, a leaf first on equal weight
                const uint64_t a0 = c < m ? A.wL[c] : kNone, a1 = c + 1 < m ? A.wL[c + 1] : kNone;
                const uint64_t b0 = ih < it ? A.wI[ih] : kNone, b1 = ih + 1 < it ? A.wI[ih + 1] : kNone;
                const uint64_t t = a0 <= b0 ? a0 + (a1 <= b0 ? a1 : b0) : b0 + (a0 <= b1 ? a0 : b1);
                uint32_t mL, mI;
                warp_upper_bound2(A.wL, c, m, A.wI, ih, it, (uint32_t)t, mL, mI);
                mL -= c;
                mI -= ih;
                if ((mL + mI) & 1) {
                    // drop the last node of the merged order: a joined node wins ties for last
                    const uint32_t lastI = mI ? A.wI[ih + mI - 1] : 0u, lastL = mL ? A.wL[c + mL - 1] : 0u;
                    const bool dropI = mI > 0 && (mL == 0 || lastI >= lastL);
                    if (dropI) mI--; else mL--;
                }
                const uint32_t pairs = (mL + mI) >> 1;
                const uint32_t *wa = A.wL + c, *wb = A.wI + ih;
                for (uint32_t j = tid; j < pairs; j += rt) {
                    // leaves among the first 2j nodes of the stable leaf-first merge:
                    // the least i with wa[i] > wb[2j - 1 - i]
                    const uint32_t p = 2 * j;
                    uint32_t lo = p > mI ? p - mI : 0, hi = p < mL ? p : mL;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (wa[mid] <= wb[p - 1 - mid]) lo = mid + 1; else hi = mid;
                    }
                    uint32_t ia = lo, ib = p - lo, wsum = 0;
                    uint32_t node[2];
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        const bool leaf = ia < mL && (ib >= mI || wa[ia] <= wb[ib]);
                        if (leaf) { node[q] = c + ia; wsum += wa[ia]; ia++; }
                        else { node[q] = m + ih + ib; wsum += wb[ib]; ib++; }
                    }
                    A.wI[it + j] = wsum;
                    A.parent[node[0]] = m + it + j;
                    A.parent[node[1]] = m + it + j;
                }
                c += mL;
                ih += mI;
                it += pairs;
                asm volatile("bar.sync 1, %0;" ::"r"(rt) : "memory");
            }
            if (tid == 0) s_rounds = round;
        }
        __syncthreads();

        // ---- lengths: parent links from each leaf to the root (joined node m - 2).
        // Large trees (their links in L2) take the joined nodes' depths round
        // by round in reverse instead: a parent is always made in a later round.
        uint32_t bad = 0;
        if (!rev) {
            const uint32_t root = 2 * m - 2;
            for (uint32_t v = tid; v < m; v += kCbThreads) {
                uint32_t d = 0, x = v;
                while (x != root && d <= HUFF_MAX_LEN) { x = A.parent[x]; d++; }
                if (d > HUFF_MAX_LEN) { bad = 1; d = HUFF_MAX_LEN; }
                A.lenS[(uint32_t)(A.keys[v] & kIdMask)] = (uint8_t)d;
            }
        } else {
            const uint32_t nI = m - 1, rounds = s_rounds;
            if (tid == 0) A.depthI[nI - 1] = 0;
            __syncthreads();
            for (int r = (int)rounds - 1; r >= 0; r--) {
                const uint32_t j0 = A.rstart[r], j1 = r + 1 < (int)rounds ? A.rstart[r + 1] : nI;
                for (uint32_t j = j0 + tid; j < j1; j += kCbThreads)
                    if (j != nI - 1) A.depthI[j] = A.depthI[A.parent[m + j] - m] + 1;
                __syncthreads();
            }
            for (uint32_t v = tid; v < m; v += kCbThreads) {
                uint32_t d = A.depthI[A.parent[v] - m] + 1;
                if (d > HUFF_MAX_LEN) { bad = 1; d = HUFF_MAX_LEN; }
                A.lenS[(uint32_t)(A.keys[v] & kIdMask)] = (uint8_t)d;
            }
        }
        if (bad) s_bad = 1;
    } else if (m == 1) {
        for (uint32_t i = tid; i < nbins; i += kCbThreads)
            if (g.hist[i]) A.lenS[i] = 1;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) set_error(g.status, HUFF_ERR_HIST_OVERFLOW);
        for (uint32_t i = tid; i < nbins; i += kCbThreads) A.lenS[i] = 0;
        __syncthreads();
    }

    // ---- canonical codewords, First, Entry, reverse codebook.  Ids are taken
    // in slices of kCbThreads; within a slice, a warp match gives each id its
    // rank among the warp's ids of equal length, and a per-length scan over
    // the warps (one warp per length, lengths 1..lmax) its rank in the slice.
    // Each warp clears and fills its own row of s_wcnt, so a slice needs two
    // barriers.  Every id's cw is written (0 when unused).
    uint32_t l_mine = 0, rank_w = 0;
    auto slice_ranks = [&](uint32_t base, uint32_t lmax) {
        __syncwarp();
        for (uint32_t l = lane; l <= lmax; l += 32) s_wcnt[warp][l] = 0;
        __syncwarp();
        const uint32_t id = base + tid;
        l_mine = id < nbins ? A.lenS[id] : 0;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, l_mine);
        rank_w = __popc(peers & ((1u << lane) - 1));
        if (rank_w == 0 && l_mine) s_wcnt[warp][l_mine] = __popc(peers);
        __syncthreads();
        for (uint32_t l = warp + 1; l <= lmax; l += kCbThreads / 32) {
            const uint32_t b = s_base[l], cnt = s_wcnt[lane][l];
            uint32_t inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= o) inc += y;
            }
            s_wcnt[lane][l] = b + inc - cnt;
            __syncwarp();
            if (lane == 31) s_base[l] = b + inc;
        }
        __syncthreads();
    };
    auto first_entry = [&]() {
        // First from the longest length down; Entry as the running count
        if (tid == 0) {
            uint32_t maxl = 0;
            for (uint32_t l = 1; l <= HUFF_MAX_LEN; l++) if (s_count[l]) maxl = l;
            s_maxlen = maxl;
            uint64_t f = 0;
            for (int l = (int)maxl - 1; l >= 1; l--) {
                f = (f + s_count[l + 1] + 1) >> 1;
                s_first[l] = f;
            }
            uint32_t e = 0;
            for (uint32_t l = 1; l < HUFF_MAX_LEN; l++) {
                e += s_count[l];
                s_entry[l + 1] = e;
            }
        }
        __syncthreads();
    };
    auto write_codes = [&](uint32_t base) {
        const uint32_t id = base + tid;
        if (l_mine) {
            const uint32_t rank = s_wcnt[warp][l_mine] + rank_w;
            cw[id] = (s_first[l_mine] + rank) | ((uint64_t)l_mine << HUFF_CW_LEN_SHIFT);
            sorted_syms[s_entry[l_mine] + rank] = id;
        } else if (id < nbins) {
            cw[id] = 0;
        }
    };
    uint64_t tb = 0;
    if (nbins <= kCbThreads) {
        // one slice: its per-length totals are the counts
        slice_ranks(0, HUFF_MAX_LEN);
        if (l_mine) tb = (uint64_t)l_mine * mycount;
        if (tid >= 1 && tid <= HUFF_MAX_LEN) s_count[tid] = s_base[tid];
        __syncthreads();
        first_entry();
        write_codes(0);
    } else {
        // one stable counting pass by length over the ids: an id's slot in
        // (length, id) order is its sorted_syms index, and slot - entry[l]
        // its rank among the codewords of length l
        auto elem = [&](uint32_t i) -> CpElem {
            const uint32_t l = A.lenS[i];
            return CpElem{l != 0, l, ((uint64_t)l << 32) | i};
        };
        // (counting by atomics: a step of ids holds many lengths, 394 against 400 us at 65,536 bins)
        cpass_count<true>(nbins, elem, s_rh, s_wsum, s_count, HUFF_MAX_LEN + 1);
        if (tid == 0) s_count[0] = 0;
        __syncthreads();
        first_entry();
        cpass_scatter(
            nbins, elem,
            [&](uint32_t slot, uint64_t pl) {
                const uint32_t l = (uint32_t)(pl >> 32), id = (uint32_t)pl;
                cw[id] = (s_first[l] + (slot - s_entry[l])) | ((uint64_t)l << HUFF_CW_LEN_SHIFT);
                sorted_syms[slot] = id;
            },
            [&](uint64_t pl) { cw[(uint32_t)pl] = 0; }, s_rh);
        for (uint32_t i = tid; i < nbins; i += kCbThreads) {
            const uint32_t l = A.lenS[i];
            if (l) tb += (uint64_t)l * g.hist[i];
        }
    }
    for (int o = 16; o; o >>= 1) tb += __shfl_xor_sync(0xFFFFFFFFu, tb, o);
    if (lane == 0 && tb) atomicAdd((unsigned long long *)&s_tbits, (unsigned long long)tb);
    __syncthreads();
    if (tid == 0) {
        hdr->nbins = nbins;
        hdr->max_len = s_maxlen;
        uint32_t nu = 0;
        for (uint32_t l = 1; l <= HUFF_MAX_LEN; l++) nu += s_count[l];
        hdr->nused = nu;
        hdr->status = overflow || s_bad ? HUFF_ERR_HIST_OVERFLOW : HUFF_OK;
        hdr->total_bits = overflow || s_bad ? 0 : s_tbits;
        hdr->nsymbols = overflow || s_bad ? 0 : s_sum;
    }
    if (tid <= HUFF_MAX_LEN) {
        hdr->first[tid] = s_first[tid];
        hdr->entry[tid] = s_entry[tid];
        hdr->count[tid] = s_count[tid];
    }
}

// ---------------------------------------------------------------- cluster form
//
// Alphabets of kCcMinBins bins or more: one thread-block cluster of CL CTAs
// (16 where the device allows it, else 8) builds the codebook.  The phases
// whose work grows with the alphabet are split over the cluster's CTAs:
//   sort      a stable LSD radix sort by count (8-bit digits); each CTA counts
//             the digits of its share of the elements, reads every CTA's digit
//             totals from distributed shared memory to find its first slot per
//             digit, and scatters its share;
//   depths    pointer jumping over the parent links (each node adds its
//             parent's distance and takes its grandparent, seven times: depths
//             up to 128), instead of one pass per round in reverse;
//   codes     each CTA counts the lengths of its id range, reads every CTA's
//             counts for First, Entry and its own base per length, and assigns
//             the codes of its ids in id order.
// A cluster barrier separates the phases.  The GenerateCL rounds stay on CTA 0:
// a round's cost is the latency of its chain (selection, co-ranking search,
// barrier), which more CTAs would lengthen by a cluster barrier per round.

namespace cg = cooperative_groups;

constexpr uint32_t kCcMinBins = 4097;      // alphabets from here on take the cluster form (their arrays
                                           // are in global memory anyway)
constexpr uint32_t kCcJumps = 7;           // pointer-jumping steps: depths up to 2^7
constexpr uint32_t kCcBigRound = 4096;     // rounds melding at least this many pairs use the whole cluster

// Scratch beyond CbArrays: parents and distances of the pointer jumping (two
// buffers each, 2m entries) and the sorted leaves' symbol ids.
__host__ __device__ inline size_t cc_extra_bytes(uint32_t nbins) {
    return 4 * align16((size_t)nbins * 8) + align16((size_t)nbins * 4);
}

__device__ __forceinline__ void cc_split(uint32_t len, uint32_t parts, uint32_t i, uint32_t &lo, uint32_t &hi) {
    lo = (uint32_t)((uint64_t)len * i / parts);
    hi = (uint32_t)((uint64_t)len * (i + 1) / parts);
}

// Segment of warp `warp` inside the CTA's element range [e0, e1).
__device__ __forceinline__ void cc_segment(uint32_t e0, uint32_t e1, uint32_t &begin, uint32_t &end) {
    const uint32_t warp = threadIdx.x >> 5, len = e1 - e0;
    const uint32_t seg = (((len + 31) / 32) + 31) & ~31u;
    begin = e0 + (warp * seg < len ? warp * seg : len);
    end = begin + seg < e1 ? begin + seg : e1;
}

struct CcShared {
    uint32_t rh[kRadixDigits][33];      // per-warp digit counts, then slots
    uint32_t tot[kRadixDigits];         // this CTA's digit totals (read by the cluster)
    uint32_t wsum[kCbThreads / 32];
    uint64_t sum;                       // this CTA's share of the histogram sum (read by the cluster)
    uint32_t used, maxc, bad;           // (read by the cluster)
    uint64_t g_sum;                     // cluster-wide values
    uint32_t g_m, g_maxc, g_bad;
    uint32_t lcnt[HUFF_MAX_LEN + 1];    // ids of each length in this CTA's range (read by the cluster)
    uint32_t count[HUFF_MAX_LEN + 1], base[HUFF_MAX_LEN + 1], entry[HUFF_MAX_LEN + 1];
    uint64_t first[HUFF_MAX_LEN + 1];
    uint32_t wcnt[kCbThreads / 32][HUFF_MAX_LEN + 1];
    uint64_t tb;                        // total bits (CTA 0 gathers the cluster's)
    uint32_t maxlen;
    uint32_t rstate[4];                 // CTA 0's round state (c, ih, it, done), read by the cluster
    uint32_t lstate[4];                 // this CTA's copy
};

// The selection of a GenerateCL round (the rule: codebook_body): the counts
// mL, mI of waiting leaves and joined nodes it melds, in pairs.  Every warp
// computes the same values from the same reads.
__device__ __forceinline__ void round_select(const CbArrays &A, uint32_t m, uint32_t c, uint32_t ih, uint32_t it,
                                             uint32_t &mL, uint32_t &mI) {
    constexpr uint64_t kNone = 1ull << 33;
    const uint64_t a0 = c < m ? A.wL[c] : kNone, a1 = c + 1 < m ? A.wL[c + 1] : kNone;
    const uint64_t b0 = ih < it ? A.wI[ih] : kNone, b1 = ih + 1 < it ? A.wI[ih + 1] : kNone;
    const uint64_t t = a0 <= b0 ? a0 + (a1 <= b0 ? a1 : b0) : b0 + (a0 <= b1 ? a0 : b1);
    warp_upper_bound2(A.wL, c, m, A.wI, ih, it, (uint32_t)t, mL, mI);
    mL -= c;
    mI -= ih;
    if ((mL + mI) & 1) {
        const uint32_t lastI = mI ? A.wI[ih + mI - 1] : 0u, lastL = mL ? A.wL[c + mL - 1] : 0u;
        const bool dropI = mI > 0 && (mL == 0 || lastI >= lastL);
        if (dropI) mI--; else mL--;
    }
}

// Melds pairs j0, j0 + stride, ... of a round (Merge Path co-ranking, leaf
// first on equal weight), recording the joined weights and parent links.
__device__ __forceinline__ void round_meld(const CbArrays &A, uint32_t m, uint32_t c, uint32_t ih, uint32_t it,
                                           uint32_t mL, uint32_t mI, uint32_t j0, uint32_t stride) {
    const uint32_t pairs = (mL + mI) >> 1;
    const uint32_t *wa = A.wL + c, *wb = A.wI + ih;
    for (uint32_t j = j0; j < pairs; j += stride) {
        const uint32_t p = 2 * j;
        uint32_t lo = p > mI ? p - mI : 0, hi = p < mL ? p : mL;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (wa[mid] <= wb[p - 1 - mid]) lo = mid + 1; else hi = mid;
        }
        uint32_t ia = lo, ib = p - lo, wsum = 0;
        uint32_t node[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const bool leaf = ia < mL && (ib >= mI || wa[ia] <= wb[ib]);
            if (leaf) { node[q] = c + ia; wsum += wa[ia]; ia++; }
            else { node[q] = m + ih + ib; wsum += wb[ib]; ib++; }
        }
        A.wI[it + j] = wsum;
        A.parent[node[0]] = m + it + j;
        A.parent[node[1]] = m + it + j;
    }
}

// One stable counting pass of the cluster: elements [0, len), CTA R owning
// [e0, e1); elem(i) gives the element (digit, payload); place(slot, payload)
// receives it at its slot in digit-major, element order.  Ends with a cluster
// barrier (every slot written).
template <typename Elem, typename Place>
__device__ void cc_pass(cg::cluster_group &cl, CcShared &S, uint32_t len, bool atomic_count, Elem elem, Place place) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t R = cl.block_rank(), CL = cl.num_blocks();
    const uint32_t lt = (1u << lane) - 1;
    uint32_t e0, e1, begin, end;
    cc_split(len, CL, R, e0, e1);
    cc_segment(e0, e1, begin, end);
    for (uint32_t i = tid; i < kRadixDigits * 33; i += kCbThreads) (&S.rh[0][0])[i] = 0;
    __syncthreads();
    for (uint32_t b = begin; b < end; b += 128) {
        CpElem e[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = b + 32 * q + lane;
            e[q] = i < end ? elem(i) : CpElem{false, 0u, 0ull};
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (atomic_count) {
                if (e[q].valid) atomicAdd(&S.rh[e[q].digit][warp], 1u);
            } else {
                const uint32_t peers = __match_any_sync(0xFFFFFFFFu, e[q].valid ? e[q].digit : 0x10000u);
                if (e[q].valid && __popc(peers & lt) == 0) S.rh[e[q].digit][warp] += __popc(peers);
            }
        }
    }
    __syncthreads();
    if (tid < kRadixDigits) {
        uint32_t t = 0;
        for (uint32_t w = 0; w < 32; w++) t += S.rh[tid][w];
        S.tot[tid] = t;
    }
    cl.sync();                                           // every CTA's totals are out
    uint32_t pre = 0, all = 0;
    if (tid < kRadixDigits) {
        for (uint32_t r = 0; r < CL; r++) {
            const uint32_t x = *cl.map_shared_rank(&S.tot[tid], r);
            all += x;
            if (r < R) pre += x;
        }
    }
    // first slot of digit d in this CTA: elements of smaller digits anywhere,
    // then this digit in the CTAs before this one
    uint32_t inc = all;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (tid < kRadixDigits && lane == 31) S.wsum[warp] = inc;
    __syncthreads();
    if (tid < kRadixDigits) {
        uint32_t wb = 0;
        for (uint32_t w = 0; w < warp; w++) wb += S.wsum[w];
        uint32_t run = wb + inc - all + pre;
        for (uint32_t w = 0; w < 32; w++) {
            const uint32_t c = S.rh[tid][w];
            S.rh[tid][w] = run;
            run += c;
        }
    }
    __syncthreads();
    for (uint32_t b = begin; b < end; b += 128) {
        CpElem e[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = b + 32 * q + lane;
            e[q] = i < end ? elem(i) : CpElem{false, 0u, 0ull};
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, e[q].valid ? e[q].digit : 0x10000u);
            const uint32_t rank = __popc(peers & lt);
            const uint32_t slot = e[q].valid ? S.rh[e[q].digit][warp] : 0u;
            __syncwarp();
            if (e[q].valid && rank == 0) S.rh[e[q].digit][warp] = slot + __popc(peers);
            __syncwarp();
            if (e[q].valid) place(slot + rank, e[q].payload);
        }
    }
    cl.sync();                                           // every slot written; totals no longer read
}

__global__ void __launch_bounds__(kCbThreads, 1) codebook_cluster_kernel(CbArgs g) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ CcShared S;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t R = cl.block_rank(), CL = cl.num_blocks();
    const uint32_t nbins = g.nbins;
    const uint32_t P = pow2_ceil(nbins);
    CbArrays A = cb_carve(g.scratch, nbins);
    uint8_t *xp = g.scratch + cb_array_bytes(nbins);
    uint32_t *jp[2], *jd[2];
    jp[0] = reinterpret_cast<uint32_t *>(xp); xp += align16((size_t)nbins * 8);
    jp[1] = reinterpret_cast<uint32_t *>(xp); xp += align16((size_t)nbins * 8);
    jd[0] = reinterpret_cast<uint32_t *>(xp); xp += align16((size_t)nbins * 8);
    jd[1] = reinterpret_cast<uint32_t *>(xp); xp += align16((size_t)nbins * 8);
    uint32_t *ids = reinterpret_cast<uint32_t *>(xp);
    huff_codebook_header *hdr = reinterpret_cast<huff_codebook_header *>(g.book);
    uint64_t *cw = reinterpret_cast<uint64_t *>(g.book + cb_cw_offset());
    uint32_t *sorted_syms = reinterpret_cast<uint32_t *>(g.book + cb_sorted_offset(nbins));

    // ---- this CTA's bins: sum, used, largest count; lengths cleared
    uint32_t b0, b1;
    cc_split(nbins, CL, R, b0, b1);
    if (tid == 0) { S.sum = 0; S.used = 0; S.maxc = 0; S.bad = 0; S.tb = 0; }
    if (tid <= HUFF_MAX_LEN) { S.lcnt[tid] = 0; S.first[tid] = 0; S.entry[tid] = 0; S.count[tid] = 0; }
    __syncthreads();
    {
        uint64_t part = 0;
        uint32_t used = 0, maxc = 0;
        for (uint32_t i = b0 + tid; i < b1; i += kCbThreads) {
            const uint32_t c = g.hist[i];
            part += c;
            used += c != 0;
            maxc = c > maxc ? c : maxc;
            A.lenS[i] = 0;
        }
        for (int o = 16; o; o >>= 1) {
            part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
            used += __shfl_xor_sync(0xFFFFFFFFu, used, o);
            maxc = max(maxc, __shfl_xor_sync(0xFFFFFFFFu, maxc, o));
        }
        if (lane == 0) {
            atomicAdd((unsigned long long *)&S.sum, (unsigned long long)part);
            atomicAdd(&S.used, used);
            atomicMax(&S.maxc, maxc);
        }
    }
    cl.sync();
    if (warp == 0) {
        uint64_t sum = 0;
        uint32_t used = 0, maxc = 0;
        if (lane < CL) {
            sum = *cl.map_shared_rank(&S.sum, lane);
            used = *cl.map_shared_rank(&S.used, lane);
            maxc = *cl.map_shared_rank(&S.maxc, lane);
        }
        for (int o = 16; o; o >>= 1) {
            sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
            used += __shfl_xor_sync(0xFFFFFFFFu, used, o);
            maxc = max(maxc, __shfl_xor_sync(0xFFFFFFFFu, maxc, o));
        }
        if (lane == 0) { S.g_sum = sum; S.g_m = used; S.g_maxc = maxc; }
    }
    __syncthreads();
    const bool overflow = S.g_sum >= (1ull << 32);
    const uint32_t m = overflow ? 0 : S.g_m;
    if (overflow && R == 0 && tid == 0) set_error(g.status, HUFF_ERR_HIST_OVERFLOW);
    uint32_t bad = 0;

    if (m >= 2) {
        // ---- sort: keys count << 32 | id, stable by count over ids in order
        const uint32_t maxcount = S.g_maxc;
        const uint32_t bits = 32 - __clz(maxcount);
        const uint32_t npass = bits > 8 ? (bits + 7) / 8 : 1;
        for (uint32_t pass = 0; pass < npass; pass++) {
            const uint32_t shift = 32 + 8 * pass;
            const uint64_t *src = A.keys + ((npass - pass) & 1) * P;
            uint64_t *dst = A.keys + ((npass - 1 - pass) & 1) * P;
            auto elem = [&](uint32_t i) -> CpElem {
                uint64_t key;
                if (pass == 0) {
                    const uint32_t c = g.hist[i];
                    key = ((uint64_t)c << 32) | i;
                    if (c == 0) return CpElem{false, 0u, key};
                } else {
                    key = src[i];
                }
                return CpElem{true, (uint32_t)(key >> shift) & (kRadixDigits - 1), key};
            };
            cc_pass(cl, S, pass == 0 ? nbins : m, pass == 0 && maxcount >= 256, elem,
                    [&](uint32_t slot, uint64_t key) { dst[slot] = key; });
        }
        {
            uint32_t k0, k1;
            cc_split(m, CL, R, k0, k1);
            for (uint32_t i = k0 + tid; i < k1; i += kCbThreads) {
                const uint64_t key = A.keys[i];
                A.wL[i] = (uint32_t)(key >> 32);
                ids[i] = (uint32_t)key;
            }
        }
        cl.sync();

        // ---- GenerateCL rounds (the rule and its proof: codebook_body).  CTA 0
        // runs the rounds that meld fewer than kCcBigRound pairs alone (their
        // cost is the latency of the round's chain); when the next round is
        // larger it publishes the state, and the whole cluster melds that
        // round, each CTA a share of the pairs, between two cluster barriers.
        {
            uint32_t c = 0, ih = 0, it = 0;
            const uint32_t rt = m <= 2048 ? 256u : (m <= 16384 ? 512u : (uint32_t)kCbThreads);
            for (;;) {
                if (R == 0 && tid < rt) {
                    while ((m - c) + (it - ih) >= 2) {
                        uint32_t mL, mI;
                        round_select(A, m, c, ih, it, mL, mI);
                        const uint32_t pairs = (mL + mI) >> 1;
                        if (pairs >= kCcBigRound && CL > 1) break;      // the cluster melds this one
                        round_meld(A, m, c, ih, it, mL, mI, tid, rt);
                        c += mL;
                        ih += mI;
                        it += pairs;
                        asm volatile("bar.sync 1, %0;" ::"r"(rt) : "memory");
                    }
                    if (tid == 0) {
                        S.rstate[0] = c;
                        S.rstate[1] = ih;
                        S.rstate[2] = it;
                        S.rstate[3] = (m - c) + (it - ih) >= 2 ? 0u : 1u;
                    }
                }
                cl.sync();                                   // CTA 0's rounds and state are out
                if (tid < 4) S.lstate[tid] = *cl.map_shared_rank(&S.rstate[tid], 0);
                __syncthreads();
                c = S.lstate[0];
                ih = S.lstate[1];
                it = S.lstate[2];
                const bool done = S.lstate[3] != 0;
                __syncthreads();
                if (done) break;
                uint32_t mL, mI;
                round_select(A, m, c, ih, it, mL, mI);
                round_meld(A, m, c, ih, it, mL, mI, R * kCbThreads + tid, CL * kCbThreads);
                c += mL;
                ih += mI;
                it += (mL + mI) >> 1;
                cl.sync();                                   // the round's nodes are out; rstate read
            }
        }

        // ---- depths by pointer jumping over the 2m - 1 nodes (root 2m - 2)
        const uint32_t nodes = 2 * m - 1, root = 2 * m - 2;
        uint32_t v0, v1;
        cc_split(nodes, CL, R, v0, v1);
        for (uint32_t v = v0 + tid; v < v1; v += kCbThreads) {
            jp[0][v] = v == root ? root : A.parent[v];
            jd[0][v] = v == root ? 0u : 1u;
        }
        cl.sync();
        uint32_t cur = 0;
        for (uint32_t k = 0; k < kCcJumps; k++) {
            const uint32_t *pc = jp[cur], *dc = jd[cur];
            uint32_t *pn = jp[cur ^ 1], *dn = jd[cur ^ 1];
            for (uint32_t v = v0 + tid; v < v1; v += kCbThreads) {
                const uint32_t p = pc[v];
                dn[v] = dc[v] + dc[p];
                pn[v] = pc[p];
            }
            cur ^= 1;
            cl.sync();
        }
        uint32_t l0, l1;
        cc_split(m, CL, R, l0, l1);
        for (uint32_t v = l0 + tid; v < l1; v += kCbThreads) {
            uint32_t d = jd[cur][v];
            if (jp[cur][v] != root || d > HUFF_MAX_LEN) { bad = 1; d = HUFF_MAX_LEN; }
            A.lenS[ids[v]] = (uint8_t)d;
        }
    } else if (m == 1) {
        for (uint32_t i = b0 + tid; i < b1; i += kCbThreads)
            if (g.hist[i]) A.lenS[i] = 1;
    }
    if (bad) atomicOr(&S.bad, 1u);
    cl.sync();                                           // lengths complete; every CTA's flag out
    if (warp == 0) {
        uint32_t any = lane < CL ? *cl.map_shared_rank(&S.bad, lane) : 0u;
        any = __any_sync(0xFFFFFFFFu, any != 0);
        if (lane == 0) S.g_bad = any;
    }
    __syncthreads();
    const bool failed = overflow || S.g_bad;
    if (S.g_bad && R == 0 && tid == 0) set_error(g.status, HUFF_ERR_HIST_OVERFLOW);

    // ---- canonical codes: lengths of this CTA's ids, then the cluster's
    // counts, First, Entry and this CTA's base per length
    for (uint32_t i = b0 + tid; i < b1; i += kCbThreads) {
        const uint32_t l = failed ? 0u : A.lenS[i];
        if (l) atomicAdd(&S.lcnt[l], 1u);
    }
    cl.sync();
    if (tid <= HUFF_MAX_LEN) {
        uint32_t all = 0, pre = 0;
        if (tid >= 1) {
            for (uint32_t r = 0; r < CL; r++) {
                const uint32_t x = *cl.map_shared_rank(&S.lcnt[tid], r);
                all += x;
                if (r < R) pre += x;
            }
        }
        S.count[tid] = all;
        S.base[tid] = pre;
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t maxl = 0;
        for (uint32_t l = 1; l <= HUFF_MAX_LEN; l++) if (S.count[l]) maxl = l;
        S.maxlen = maxl;
        uint64_t f = 0;
        for (int l = (int)maxl - 1; l >= 1; l--) {
            f = (f + S.count[l + 1] + 1) >> 1;
            S.first[l] = f;
        }
        uint32_t e = 0;
        for (uint32_t l = 1; l < HUFF_MAX_LEN; l++) {
            e += S.count[l];
            S.entry[l + 1] = e;
        }
    }
    __syncthreads();
    // slices of kCbThreads ids: a warp match ranks each id among the warp's ids
    // of its length, a per-length scan over the warps (S.base carries the
    // running base) gives its rank among this CTA's ids of that length
    uint64_t tb = 0;
    for (uint32_t sb = b0; sb < b1; sb += kCbThreads) {
        __syncwarp();
        for (uint32_t l = lane; l <= HUFF_MAX_LEN; l += 32) S.wcnt[warp][l] = 0;
        __syncwarp();
        const uint32_t id = sb + tid;
        const uint32_t lm = id < b1 && !failed ? A.lenS[id] : 0u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, lm);
        const uint32_t rank_w = __popc(peers & ((1u << lane) - 1));
        if (rank_w == 0 && lm) S.wcnt[warp][lm] = __popc(peers);
        __syncthreads();
        for (uint32_t l = warp + 1; l <= S.maxlen; l += kCbThreads / 32) {
            const uint32_t bl = S.base[l], cnt = S.wcnt[lane][l];
            uint32_t inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= o) inc += y;
            }
            S.wcnt[lane][l] = bl + inc - cnt;
            __syncwarp();
            if (lane == 31) S.base[l] = bl + inc;
        }
        __syncthreads();
        if (lm) {
            const uint32_t rank = S.wcnt[warp][lm] + rank_w;
            cw[id] = (S.first[lm] + rank) | ((uint64_t)lm << HUFF_CW_LEN_SHIFT);
            sorted_syms[S.entry[lm] + rank] = id;
            tb += (uint64_t)lm * g.hist[id];
        } else if (id < b1) {
            cw[id] = 0;
        }
        __syncthreads();
    }
    for (int o = 16; o; o >>= 1) tb += __shfl_xor_sync(0xFFFFFFFFu, tb, o);
    if (lane == 0 && tb) atomicAdd((unsigned long long *)cl.map_shared_rank(&S.tb, 0), (unsigned long long)tb);
    cl.sync();                                           // every CTA's bits are in; no remote access after this
    if (R == 0) {
        if (tid == 0) {
            hdr->nbins = nbins;
            hdr->max_len = S.maxlen;
            uint32_t nu = 0;
            for (uint32_t l = 1; l <= HUFF_MAX_LEN; l++) nu += S.count[l];
            hdr->nused = nu;
            hdr->status = failed ? HUFF_ERR_HIST_OVERFLOW : HUFF_OK;
            hdr->total_bits = failed ? 0 : S.tb;
            hdr->nsymbols = failed ? 0 : S.g_sum;
        }
        if (tid <= HUFF_MAX_LEN) {
            hdr->first[tid] = S.first[tid];
            hdr->entry[tid] = S.entry[tid];
            hdr->count[tid] = S.count[tid];
        }
    }
}

__global__ void __launch_bounds__(kCbThreads, 1) codebook_kernel(CbArgs g) {
    extern __shared__ __align__(16) uint8_t smem[];
    codebook_body<false>(g, g.nbins <= kCbSmemBins ? smem : g.scratch);
}

// Alphabets above 65,536 bins (arrays in the global scratch).
__global__ void __launch_bounds__(kCbThreads, 1) codebook_big_kernel(CbArgs g) {
    codebook_body<true>(g, g.scratch);
}

// Codebooks of a batch: CTA b builds those of fields b, b + grid, ...;
// alphabets above the shared-memory limit use scratch + b * scratch_stride.
__global__ void __launch_bounds__(kCbThreads, 1) codebook_batch_kernel(const CbArgs *gs, uint32_t nfields,
                                                                     uint8_t *scratch, size_t scratch_stride) {
    extern __shared__ __align__(16) uint8_t smem[];
    for (uint32_t f = blockIdx.x; f < nfields; f += gridDim.x) {
        const CbArgs g = gs[f];
        codebook_body<false>(g, g.nbins <= kCbSmemBins ? smem : scratch + blockIdx.x * scratch_stride);
        __syncthreads();     // the next field reuses the shared state
    }
}

size_t codebook_array_bytes(uint32_t nbins) { return cb_array_bytes(nbins); }

// Shared memory a batched codebook launch needs when its largest alphabet is max_nbins.
size_t codebook_batch_smem(uint32_t max_nbins) { return max_nbins <= kCbSmemBins ? cb_array_bytes(max_nbins) : 0; }

huff_status codebook_batch_prepare(uint32_t max_nbins, int *ctas_per_sm) {
    const size_t smem = codebook_batch_smem(max_nbins);
    if (!allow_dynamic_smem((const void *)codebook_batch_kernel, smem))
        return HUFF_ERR_CUDA;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, codebook_batch_kernel, kCbThreads, smem);
    *ctas_per_sm = occ < 1 ? 1 : occ;
    return HUFF_OK;
}

huff_status codebook_batch_launch(const CbArgs *d_args, uint32_t nfields, uint32_t max_nbins, uint32_t grid,
                                  uint8_t *scratch, size_t scratch_stride, cudaStream_t st) {
    codebook_batch_kernel<<<grid, kCbThreads, codebook_batch_smem(max_nbins), st>>>(d_args, nfields, scratch,
                                                                                     scratch_stride);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

size_t codebook_scratch_bytes(uint32_t nbins) {
    if (nbins >= kCcMinBins) return cb_array_bytes(nbins) + cc_extra_bytes(nbins);
    return nbins <= kCbSmemBins ? 0 : cb_array_bytes(nbins);
}

// Cluster size for the cluster form on the current device: 16 where a
// 16-CTA cluster of the kernel fits, else 8 (0: no cluster launch possible).
static int cluster_size() {
    static int cached[64];
    static bool known[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (known[dev]) return cached[dev];
    int best = 0;
    for (int cl : {16, 8}) {
        if (cl == 16 && cudaFuncSetAttribute(codebook_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                             1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(kCbThreads);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, codebook_cluster_kernel, &cfg) == cudaSuccess && n >= 1) {
            best = cl;
            break;
        }
        cudaGetLastError();
    }
    cached[dev] = best;
    known[dev] = true;
    return best;
}

huff_status codebook_launch(const uint32_t *d_hist, uint32_t nbins, void *d_codebook, uint8_t *scratch,
                            uint32_t *status, cudaStream_t st) {
    CbArgs a;
    a.hist = d_hist;
    a.nbins = nbins;
    a.book = static_cast<uint8_t *>(d_codebook);
    a.scratch = scratch;
    a.status = status;
    if (nbins >= kCcMinBins) {
        const int cl = cluster_size();
        if (cl > 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cl);
            cfg.blockDim = dim3(kCbThreads);
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cl;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            if (cudaLaunchKernelEx(&cfg, codebook_cluster_kernel, a) != cudaSuccess) return HUFF_ERR_CUDA;
            note_launch();
            return HUFF_OK;
        }
    }
    if (nbins > kSmallAlphabet) {
        codebook_big_kernel<<<1, kCbThreads, 0, st>>>(a);
        note_launch();
        return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
    }
    size_t smem = nbins <= kCbSmemBins ? cb_array_bytes(nbins) : 0;
    if (!allow_dynamic_smem((const void *)codebook_kernel, smem))
        return HUFF_ERR_CUDA;
    codebook_kernel<<<1, kCbThreads, smem, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

}  // namespace huff
