// Segment encoder: Sec. IV-C reduce-merge and the placement that replaces the
// shuffle-merge steps.  Codewords of at most 23 bits fit the 32-bit table
// entry; a longer one (rare: the field's least frequent symbols) has a flag
// entry, and a segment that meets one takes its runs from the codebook's
// 64-bit codewords instead.
//
// Every merge thread owns one contiguous segment of each tile: NV consecutive
// 16-byte vectors of the staged tile (NV odd, so the 16-byte loads of eight
// neighbouring lanes fall in eight different bank groups).  Per tile:
//  * reduce-merge: the segment's symbols are looked up and concatenated, 2^r
//    at a time, into runs of at most 64 bits held in registers;
//  * one scan over the CTA: a warp shuffle scan of the segment lengths (and of
//    each segment's last 32 bits), then the 8 warp totals; this gives every
//    segment its bit position in the tile and the bits that precede it in its
//    first word;
//  * placement: each thread appends its runs to the tile's words in a shared
//    bit ring with plain stores, starting with its first word completed from
//    the predecessor's bits; the word a segment shares with the next one is
//    left to that segment.  Every ring word of the tile is stored exactly
//    once: no shared-memory atomics, no zeroing.
// The tile's length and last 32 bits are published for the decoupled
// look-back right after the scan, before the placement.  Four helper warps
// (one per SM sub-partition, so that their work loads the schedulers evenly)
// take every fourth tile each: a decoupled look-back over 128 predecessors per
// step for its stream offset, then the copy of its words from the ring into
// the dense stream.
//
// Fields this path does not take (a chunk-aligned layout, a tile that could
// outgrow the ring) run the general encoder in the same launch; the choice is
// made on the device from the codebook header.
#pragma once

#include "encode_impl.cuh"

namespace huff {

// Vectors per segment, bulk-copy stages and bit-ring words per symbol width.
// The ring holds the tiles that wait for their stream offsets and must hold a
// worst-case tile (every codeword of the longest length the path takes); more
// vectors per segment spread the per-tile work over more symbols.
template <typename Sym>
struct SegGeom;
template <>
struct SegGeom<uint8_t> {
    static constexpr int NV = 3;
    static constexpr int NST = 3;
    static constexpr uint32_t RW = 16384;
};
#ifndef HUFF_SEG_NV16
#define HUFF_SEG_NV16 7
#endif
#ifndef HUFF_SEG_NST16
#define HUFF_SEG_NST16 2
#endif
#ifndef HUFF_SEG_RW16
#define HUFF_SEG_RW16 12288
#endif
template <>
struct SegGeom<uint16_t> {
    static constexpr int NV = HUFF_SEG_NV16;
    static constexpr int NST = HUFF_SEG_NST16;
    static constexpr uint32_t RW = HUFF_SEG_RW16;
};
template <>
struct SegGeom<uint32_t> {
    static constexpr int NV = 5;
    static constexpr int NST = 2;
    static constexpr uint32_t RW = 8192;
};

#ifndef HUFF_SEG_SLOTS
#define HUFF_SEG_SLOTS 8
#endif
constexpr int kSegSlots = HUFF_SEG_SLOTS;  // tiles between merge and write-out
constexpr uint32_t kSegEntryLen = 23;      // longest codeword of the 32-bit table entry
constexpr uint32_t kLong32 = 1u << 6;      // table entry of a longer codeword (bits 5..8 of an entry are free)
constexpr uint32_t kSegMaxLen = kEncMaxLen;   // the ring's worst-case tile bounds it further
constexpr uint32_t kSegRingPad = 32;       // words after the ring: the copy reads one word past a tile
constexpr int kSegMaxStages = 4;
#ifndef HUFF_SEG_HELPERS
#define HUFF_SEG_HELPERS 4
#endif
constexpr int kSegHelpers = HUFF_SEG_HELPERS;   // look-back + write-out warps
constexpr int kLbPer = 4;                  // descriptors per lane per look-back step (128 per warp)
constexpr int kSegThreads = kEncThreads + 32 * kSegHelpers;
constexpr int kSegCoff = 32;               // chunk offsets per tile kept in shared memory

template <typename Sym>
__host__ __device__ constexpr uint32_t seg_lane_bytes() { return SegGeom<Sym>::NV * 16u; }
template <typename Sym>
__host__ __device__ constexpr uint32_t seg_lane_syms() { return seg_lane_bytes<Sym>() / (uint32_t)sizeof(Sym); }
template <typename Sym>
__host__ __device__ constexpr uint32_t seg_sub_bytes() { return kEncThreads * seg_lane_bytes<Sym>(); }
template <typename Sym>
__host__ __device__ constexpr uint32_t seg_sub_syms() { return kEncThreads * seg_lane_syms<Sym>(); }

// Reduction factors of the segment path: a run stays inside one vector, and
// at most 12 runs per segment are held in registers.
template <typename Sym>
__host__ __device__ constexpr int seg_r_min() { return sizeof(Sym) == 4 ? 1 : 2; }
template <typename Sym>
__host__ __device__ constexpr int seg_r_max() { return sizeof(Sym) == 1 ? 4 : sizeof(Sym) == 2 ? 3 : 2; }

// Dynamic shared memory of the segment path: stages, bit ring, table.
template <typename Sym>
__host__ __device__ inline size_t seg_smem_bytes(uint32_t tslots, bool gtab) {
    return (size_t)SegGeom<Sym>::NST * seg_sub_bytes<Sym>() + (SegGeom<Sym>::RW + kSegRingPad) * 4ull +
           (gtab ? 0 : ((4ull * tslots + 127) & ~127ull));
}

// Tiles span at most kSegCoff chunk starts: their chunk offsets go through
// shared memory (else straight to global memory, fixed up by the write-out).
template <typename Sym>
__host__ __device__ inline bool seg_coff_smem(int chunk_log2) {
    return (seg_sub_syms<Sym>() >> chunk_log2) + 1 <= (uint32_t)kSegCoff;
}

// The path takes a codebook whose worst-case tile (every codeword max_len
// bits) fits the ring: up to 27 bits for u16 symbols, 42 for u8, 48 for u32.
template <typename Sym>
__host__ __device__ inline bool seg_fits(uint32_t max_len) {
    return max_len >= 1 && max_len <= kSegMaxLen &&
           (uint64_t)seg_sub_syms<Sym>() * max_len + 64 <= SegGeom<Sym>::RW * 32ull;
}

static_assert(kSegSlots % kSegHelpers == 0, "slots per helper warp");

struct SegShared {
    uint64_t bars[kSegMaxStages];        // stages (bulk copies)
    uint64_t full[kSegSlots];            // merge -> helper: length and last bits published
    uint64_t done[kSegSlots];            // merge -> helper: the tile's ring words stored (256 arrivals)
    uint64_t sfree[kSegSlots];           // write-out -> merge: slot reusable
    uint32_t stage_tile[kSegMaxStages];
    TileSlot slot[kSegSlots];            // pad = ring words allocated to the tile
    uint32_t ring_tail;                  // ring words before this counter are free again
    uint32_t wdone;                      // tiles written out (in order)
    uint32_t wlen[2][kEncThreads / 32];  // warp totals of the segment lengths (double-buffered)
    uint32_t wtail[2][kEncThreads / 32]; // the warps' last 32 bits
    uint32_t coff[kSegSlots][kSegCoff];  // chunk offsets relative to the tile
    EncField f0;
    uint32_t stage_field[kSegMaxStages]; // batched form: the field of each stage's tile
};

// The segment path's table entry of a codeword: the 32-bit entry up to 23
// bits, kLong32 above, kBad32 for none.
__device__ __forceinline__ uint32_t seg_entry_from_cw(uint64_t c) {
    const uint32_t l = (uint32_t)(c >> HUFF_CW_LEN_SHIFT);
    return l > kSegEntryLen ? kLong32 : entry_from_cw<uint32_t>(c);
}

// Shared-memory accesses by 32-bit shared-window address.  The table is
// read-only once loaded, so its loads may be scheduled freely; stage loads
// and ring stores are ordered with the waits around them.
__device__ __forceinline__ uint32_t lds_tab(uint32_t a) {
    uint32_t v;
    asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint4 lds_v4(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ void sts_if(bool p, uint32_t a, uint32_t v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.u32 [%0], %1;\n\t}"
                 ::"r"(a), "r"(v), "r"((uint32_t)p) : "memory");
}

// Appends a run of rb (0..64) bits, right-aligned in hi:lo, after the e5 bits
// already in the word at shared address wa (held in cur, left-aligned).  The
// run is shifted so that it ends at its end position: f0 is the word holding
// that position, f1 and f2 the two before; the first of them is merged into
// cur.  Completed words are stored; the partial last word stays in cur.
__device__ __forceinline__ void seg_put(uint32_t &cur, uint32_t &e5, uint32_t &wa, uint32_t hi, uint32_t lo,
                                        uint32_t rb) {
    const uint32_t t = e5 + rb;            // 0..95
    const uint32_t t5 = t & 31u;
    const uint32_t s = 32u - t5;           // 1..32 (a shift of 32 moves a whole word)
    const uint32_t f0 = __funnelshift_lc(0u, lo, s);
    const uint32_t f1 = __funnelshift_lc(lo, hi, s);
    const uint32_t f2 = __funnelshift_lc(hi, 0u, s);
    const bool p1 = t >= 32u, p2 = t >= 64u;
    const uint32_t w0 = cur | (p2 ? f2 : (p1 ? f1 : f0));
    sts_if(p1, wa, w0);
    sts_if(p2, wa + 4, f1);
    cur = p1 ? f0 : w0;
    wa += (t >> 5) << 2;
    e5 = t5;
}

struct SegPut {
    uint32_t cur, e5, wa;
};

// A run longer than 64 bits (rare: 2^r codewords of above 64 / 2^r bits on
// average), codeword by codeword; symbols from global memory, since the stage
// may be refilled already; flagged entries take the 64-bit codeword.  Out of
// line, so the common path keeps its registers.
template <typename Sym, int TAB>
__device__ __noinline__ SegPut seg_put_long(SegPut st, const Sym *symp, uint64_t first, int count, uint64_t n,
                                            const uint32_t *gtab, uint32_t tab_s, uint32_t nbins, uint32_t tmask,
                                            const uint64_t *gcw) {
    for (int x = 0; x < count; x++) {
        const uint64_t i = first + x;
        if (i >= n) break;
        const uint32_t sy = (uint32_t)symp[i];
        const uint32_t en = TAB == 2 ? (sy < nbins ? __ldg(gtab + sy) : kBad32) : lds_tab(tab_s + ((sy & tmask) << 2));
        if ((en & kLong32) && sy < nbins) {            // (a symbol out of range is an error already)
            const uint64_t cw = gcw[sy];
            const uint32_t l = (uint32_t)(cw >> HUFF_CW_LEN_SHIFT);
            const uint64_t code = cw & ((1ull << l) - 1);
            seg_put(st.cur, st.e5, st.wa, (uint32_t)(code >> 32), (uint32_t)code, l);
        } else {
            const uint32_t l = en & 31u;
            seg_put(st.cur, st.e5, st.wa, 0u, l ? en >> (32u - l) : 0u, l);
        }
    }
    return st;
}

// Reduce-merge of one vector's symbols into runs of 2^R2 codewords:
// (hi:lo) the run right-aligned, rb its length; every entry is OR-ed into bad
// (kBad32 marks a symbol without codeword).  FULL: all symbols valid.
template <typename Sym, int TAB, int R2, bool FULL>
__device__ __forceinline__ void seg_vec_runs(const uint32_t *sv, uint32_t valid, const uint32_t *gtab, uint32_t tab_s,
                                             uint32_t nbins, uint32_t tmask, uint32_t *hi, uint32_t *lo, uint32_t *rb,
                                             uint32_t &bad) {
    constexpr int V = VecOf<Sym>::N;
    constexpr int RL = 1 << R2;
    constexpr int NRV = V / RL;
#pragma unroll
    for (int r = 0; r < NRV; r++) {
        uint32_t e[RL];
#pragma unroll
        for (int x = 0; x < RL; x++) {
            const int xi = r * RL + x;
            uint32_t en = TAB == 2 ? (sv[xi] < nbins ? __ldg(gtab + sv[xi]) : kBad32)
                                   : lds_tab(tab_s + ((sv[xi] & tmask) << 2));
            if (!FULL && xi >= (int)valid) en = 0u;       // past n: length 0
            e[x] = en;
        }
        uint32_t h = 0, l = 0, es = 0, eo = 0;
#pragma unroll
        for (int x = 0; x < RL; x++) {
            h = __funnelshift_l(l, h, e[x]);
            l = __funnelshift_l(e[x], l, e[x]);
            es += e[x];
            eo |= e[x];
        }
        bad |= eo;
        hi[r] = h;
        lo[r] = l;
        rb[r] = es & 511u;
    }
}

// Bulk-copy producer of the segment path (merge thread 0): every stage holds
// one tile; tile ids are taken one ahead.
struct SegProducer {
    uint32_t next;
    uint32_t slot;
};

// Batched form: the field of segment tile g, from the first tile ids
// (sfirst[0] = 0 <= g < sfirst[nf]; fields without tiles are passed over).
__device__ __forceinline__ uint32_t seg_field_of(const uint32_t *sfirst, uint32_t nf, uint32_t g) {
    uint32_t lo = 0, hi = nf;              // sfirst[lo] <= g < sfirst[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (sfirst[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename Sym, bool BATCH>
__device__ __forceinline__ void seg_produce(const EncArgs &a, SegProducer &p, uint32_t total, uint8_t *stage,
                                            SegShared &T, const uint32_t *sfirst) {
    constexpr uint32_t SUB = seg_sub_syms<Sym>();
    constexpr uint32_t SUBB = seg_sub_bytes<Sym>();
    constexpr int NST = SegGeom<Sym>::NST;
    uint32_t g = total;
    if (p.next < total) {
        g = p.next;
        p.next = take_tile(a);             // not waited on until the next call
    }
    const int s = (int)(p.slot % NST);
    reinterpret_cast<volatile uint32_t *>(T.stage_tile)[s] = g;
    if (g < total) {
        const uint8_t *sym = a.one.sym;
        uint64_t n = a.one.n, j = g;
        bool aligned = a.one.aligned;
        if constexpr (BATCH) {
            const uint32_t f = seg_field_of(sfirst, a.nfields, g);
            reinterpret_cast<volatile uint32_t *>(T.stage_field)[s] = f;
            const EncField &F = a.fields[f];
            sym = F.sym;
            n = F.n;
            aligned = F.aligned;
            j = g - sfirst[f];
        }
        const uint64_t s0 = j * SUB;
        if (aligned && s0 + SUB <= n) {
            mbar_arrive_expect_tx(&T.bars[s], SUBB);
            bulk_g2s(stage + s * SUBB, sym + s0 * sizeof(Sym), SUBB, &T.bars[s]);
        } else {
            mbar_arrive(&T.bars[s]);
        }
    }
    p.slot++;
}

// The 8 merge warps of the segment path.  TAB 0: codebook entries in shared
// memory (tab[s & tmask]); TAB 2: the 32-bit entries in global memory.  MANY:
// chunks shorter than a segment (several chunk boundaries per segment).
// BATCH: tiles of many fields (sfirst: their first tile ids; TAB 2 with each
// field's own entries); the field's values are read per tile.  LONG: some
// codeword has more than 23 bits (flag entries).
template <typename Sym, int TAB, int R2, bool MANY, bool BATCH, bool LONG>
__device__ __forceinline__ void seg_merge(const EncArgs &a, uint8_t *stage, uint32_t *ring, const uint32_t *tab,
                                          uint32_t total, SegShared &T, const uint32_t *sfirst) {
    constexpr int V = VecOf<Sym>::N;
    constexpr int NV = SegGeom<Sym>::NV;
    constexpr int NST = SegGeom<Sym>::NST;
    constexpr int RL = 1 << R2;
    constexpr int NRV = V / RL;            // runs per vector
    constexpr int NR = NV * NRV;           // runs per segment
    constexpr uint32_t SEG = seg_lane_syms<Sym>();
    constexpr uint32_t SUB = seg_sub_syms<Sym>();
    constexpr uint32_t SUBB = seg_sub_bytes<Sym>();
    constexpr uint32_t RW = SegGeom<Sym>::RW;
    constexpr int NW = kEncThreads / 32;
    static_assert(RL <= V, "a run stays inside one vector");
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t tmask = a.tslots - 1;
    // the field's values (per tile in a batched launch)
    uint64_t n = a.one.n;
    uint32_t nbins = a.one.nbins;
    const Sym *symp = reinterpret_cast<const Sym *>(a.one.sym);
    uint32_t *status = a.one.status;
    int M = a.one.chunk_log2;
    uint32_t cmask = (1u << M) - 1;                  // M <= 30
    uint64_t *offs = a.one.offs;
    bool faligned = a.one.aligned;
    bool csm = seg_coff_smem<Sym>(M);
    const uint8_t *bookp = a.one.book;
    if constexpr (BATCH) status = a.fields[0].status;
    volatile uint32_t *stage_tile = T.stage_tile;
    const uint32_t stage_s = smem_u32(stage), ring_s = smem_u32(ring);
    const uint32_t tab_s = TAB == 2 ? 0u : smem_u32(tab);
    const uint32_t rmask = sizeof(Sym) == 1 ? ~(tmask * 0x01010101u)
                           : sizeof(Sym) == 2 ? ~(tmask | (tmask << 16)) : ~tmask;

    SegProducer prod{0u, 0u};
    if (tid == 0) {
        prod.next = take_tile(a);
        for (int i = 0; i < NST; i++) seg_produce<Sym, BATCH>(a, prod, total, stage, T, sfirst);
    }
    merge_sync();

    uint32_t head = 0;                     // ring words allocated so far (running counter)
    uint32_t s = 0, sph = 0;               // stage of tile t and its mbarrier phase parity
    volatile uint32_t *ring_tail = &T.ring_tail;
    for (uint32_t t = 0;; t++) {
        const uint32_t g = stage_tile[s];
        const uint32_t sl = t % kSegSlots;
        if (t >= (uint32_t)kSegSlots && !mbar_wait_bounded(&T.sfree[sl], ((t / kSegSlots) - 1) & 1))
            set_error(status, HUFF_ERR_TIMEOUT);
        if (g >= total) {
            // no more tiles: one end mark for the next tile of each helper
            if (tid == 0) {
                for (uint32_t k = 0; k < (uint32_t)kSegHelpers; k++) {
                    const uint32_t tk = t + k, sk = tk % kSegSlots;
                    if (k > 0 && tk >= (uint32_t)kSegSlots &&
                        !mbar_wait_bounded(&T.sfree[sk], ((tk / kSegSlots) - 1) & 1))
                        set_error(status, HUFF_ERR_TIMEOUT);
                    T.slot[sk].g = 0xFFFFFFFFu;
                    mbar_arrive(&T.full[sk]);
                }
            }
            break;
        }
        uint32_t j = g;                                         // the tile within its field
        uint32_t fld = 0;
        if constexpr (BATCH) {
            fld = reinterpret_cast<volatile uint32_t *>(T.stage_field)[s];
            const EncField &Fb = a.fields[fld];
            j = g - sfirst[fld];
            n = Fb.n;
            nbins = Fb.nbins;
            symp = reinterpret_cast<const Sym *>(Fb.sym);
            status = Fb.status;
            M = Fb.chunk_log2;
            cmask = (1u << M) - 1;
            offs = Fb.offs;
            faligned = Fb.aligned;
            csm = seg_coff_smem<Sym>(M);
            tab = Fb.etab;
            bookp = Fb.book;
        }
        if (!mbar_wait_bounded(&T.bars[s], sph)) set_error(status, HUFF_ERR_TIMEOUT);
        // symbol indices fit 32 bits (n < 2^32)
        const uint32_t s0 = j * SUB;
        const bool full = faligned && (uint64_t)s0 + SUB <= n;
        const uint32_t q0 = s0 + tid * SEG;                     // first symbol of this segment

        // ---- reduce-merge of the segment into NR runs
        uint32_t hi[NR], lo[NR], rb[NR];
        uint32_t bad = 0;
        bool oot = false;                                       // a symbol beyond the shared table
        if (full) {
            const uint32_t sp = stage_s + s * SUBB + tid * (NV * 16);
            uint32_t rng = 0;
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const uint4 vec = lds_v4(sp + 16 * v);
                if (TAB == 0) rng |= vec.x | vec.y | vec.z | vec.w;
                uint32_t sv[V];
                sym_from_vec(vec, sv, Sym());
                seg_vec_runs<Sym, TAB, R2, true>(sv, V, tab, tab_s, nbins, tmask, hi + v * NRV, lo + v * NRV,
                                                 rb + v * NRV, bad);
            }
            oot = TAB == 0 && (rng & rmask) != 0;
        } else {
            uint32_t rng = 0;
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const uint64_t i0 = q0 + (uint64_t)v * V;
                const uint32_t vl = i0 >= n ? 0u : (n - i0 < (uint64_t)V ? (uint32_t)(n - i0) : (uint32_t)V);
                uint32_t sv[V];
#pragma unroll
                for (int x = 0; x < V; x++) {
                    sv[x] = x < (int)vl ? (uint32_t)symp[i0 + x] : 0u;
                    rng |= sv[x];
                }
                seg_vec_runs<Sym, TAB, R2, false>(sv, vl, tab, tab_s, nbins, tmask, hi + v * NRV, lo + v * NRV,
                                                  rb + v * NRV, bad);
            }
            oot = TAB == 0 && (rng & ~tmask) != 0;
        }
        if ((bad & kBad32) || oot) {
            // a symbol without codeword, or out of range: find out which
            uint32_t code = HUFF_ERR_NOT_IN_CODEBOOK;
            for (uint32_t x = 0; x < SEG; x++) {
                const uint64_t i = q0 + x;
                if (i < n && (uint32_t)symp[i] >= nbins) code = HUFF_ERR_SYMBOL_RANGE;
            }
            set_error(status, code);
        }
        if (LONG && (bad & kLong32)) {
            // a codeword over 23 bits: this segment's runs from the codebook's
            // 64-bit codewords (the last 64 bits of each run, and its length)
            const uint64_t *gcw = reinterpret_cast<const uint64_t *>(bookp + cb_cw_offset());
#pragma unroll
            for (int q = 0; q < NR; q++) {
                uint64_t acc = 0;
                uint32_t len = 0;
#pragma unroll
                for (int x = 0; x < RL; x++) {
                    const uint64_t i = q0 + (uint64_t)(q * RL + x);
                    if (i < n) {
                        const uint32_t sy = (uint32_t)symp[i];
                        const uint64_t cw = sy < nbins ? gcw[sy] : 0ull;
                        const uint32_t l = (uint32_t)(cw >> HUFF_CW_LEN_SHIFT);
                        acc = (acc << l) | (cw & ((1ull << l) - 1));
                        len += l;
                    }
                }
                hi[q] = (uint32_t)(acc >> 32);
                lo[q] = (uint32_t)acc;
                rb[q] = len;
            }
        }

        // ---- the segment's length and last 32 bits
        uint32_t L = 0, tail = 0;
#pragma unroll
        for (int q = 0; q < NR; q++) {
            L += rb[q];
            tail = __funnelshift_lc(0u, tail, rb[q]) | lo[q];
        }
        // ---- one scan: warp shuffles, then the warp totals
        // A segment of a full tile holds at least 32 bits when it has 32 or
        // more symbols (every codeword has a bit), so its own last 32 bits are
        // what the next segment needs; otherwise they are combined.
        const bool tscan = SEG < 32 || !full;
        uint32_t inc = L, ct = tail;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (tscan) {
                const uint32_t pt = __shfl_up_sync(0xFFFFFFFFu, ct, o);
                if (lane >= (uint32_t)o) ct = __funnelshift_lc(0u, pt, inc) | ct;
            }
            if (lane >= (uint32_t)o) inc += y;
        }
        const uint32_t pb = t & 1;
        if (lane == 31) {
            T.wlen[pb][warp] = inc;
            T.wtail[pb][warp] = ct;
        }
        // the bits before this segment within its warp (none for lane 0)
        uint32_t ptail = __shfl_up_sync(0xFFFFFFFFu, ct, 1);
        if (lane == 0) ptail = 0;
        merge_sync();
        // every merge thread has read stage s: refill it
        if (tid == 0) seg_produce<Sym, BATCH>(a, prod, total, stage, T, sfirst);
        const uint32_t wl = lane < (uint32_t)NW ? T.wlen[pb][lane] : 0u;
        const uint32_t wt = lane < (uint32_t)NW ? T.wtail[pb][lane] : 0u;
        uint32_t wi = wl;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= (uint32_t)o) wi += y;
        }
        const uint32_t wbase = __shfl_sync(0xFFFFFFFFu, wi - wl, warp);
        const uint32_t Lt = __shfl_sync(0xFFFFFFFFu, wi, NW - 1);
        uint32_t wpred, last32;
        if (full) {
            // every warp of a full tile holds at least 32 bits
            wpred = __shfl_sync(0xFFFFFFFFu, wt, (warp + NW - 1) % NW);
            if (warp == 0) wpred = 0;
            last32 = __shfl_sync(0xFFFFFFFFu, wt, NW - 1);
        } else {
            uint32_t cw = 0;
            wpred = 0;
#pragma unroll
            for (int w2 = 0; w2 < NW; w2++) {
                if ((uint32_t)w2 == warp) wpred = cw;
                cw = __funnelshift_lc(0u, cw, __shfl_sync(0xFFFFFFFFu, wl, w2)) | __shfl_sync(0xFFFFFFFFu, wt, w2);
            }
            last32 = cw;
        }
        // ... completed with the earlier warps' bits: all a segment needs when
        // its predecessors in the warp hold fewer than 32 bits (combined tails);
        // otherwise only lane 0 takes them
        if (tscan) ptail = __funnelshift_lc(0u, wpred, inc - L) | ptail;
        else if (lane == 0) ptail = wpred;
        const uint32_t pos = wbase + inc - L;                   // tile bit of the segment's first bit

        // ---- ring words for the tile; publish its length and last bits
        const uint32_t Lw = (Lt + 31) >> 5;
        const bool room = Lw <= RW;                             // false only with symbols without codeword
        const uint32_t Wa = room ? Lw : 0u;
        if (head % RW + Wa > RW) head += RW - head % RW;       // tiles do not wrap
        if (tid == 0) {
            if (!room) set_error(status, HUFF_ERR_NOT_IN_CODEBOOK);
            st_relaxed_u64(&a.desc[2 * (uint64_t)g], kFlagAgg | ((uint64_t)last32 << 24) | Lt);
            if (j == 0) st_relaxed_u64(&a.desc[2 * (uint64_t)g + 1], kFlagPre | Lt);   // a field's first tile
            T.slot[sl].g = g;
            T.slot[sl].f = fld;
            T.slot[sl].j = j;
            T.slot[sl].L = Lt;
            T.slot[sl].base = head;
            T.slot[sl].pad = Wa;
            mbar_arrive(&T.full[sl]);
        }
        {
            // room in the ring (freed by the write-out)
            uint32_t spins = 0;
            while (head + Wa - *ring_tail > RW) {
                if (++spins > kSpinLimit) {
                    set_error(status, HUFF_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(256);
            }
            __threadfence_block();
        }

        // ---- chunk offsets (relative to the tile; the write-out adds its offset)
        if constexpr (!MANY) {
            // at most one chunk boundary in this segment: chunk c, before run qb
            const uint32_t qoff = q0 & cmask;
            const uint32_t qb = (((cmask + 1u) - qoff) & cmask) >> R2;
            uint32_t cpos = pos;
#pragma unroll
            for (int q = 0; q < NR; q++)
                if ((uint32_t)q < qb) cpos += rb[q];
            const uint32_t c = (q0 >> M) + (qoff ? 1u : 0u);
            if (qb < (uint32_t)NR && ((uint64_t)c << M) < n) {
                if (csm) T.coff[sl][c - ((s0 >> M) + ((s0 & cmask) ? 1u : 0u))] = cpos;
                else offs[c] = cpos;
            }
        }

        // ---- placement: the segment's runs, word by word, plain stores
        if (room) {
            const uint32_t tb = ring_s + ((head % RW) << 2);       // the tile's first word
            uint32_t wa = tb + ((pos >> 5) << 2);
            uint32_t e5 = pos & 31u;
            uint32_t cur = __funnelshift_lc(0u, ptail, 32u - e5);   // the predecessor's bits of this word
#pragma unroll
            for (int q = 0; q < NR; q++) {
                if (MANY) {
                    const uint64_t i = q0 + ((uint64_t)q << R2);
                    if ((i & cmask) == 0 && i < n) offs[i >> M] = ((wa - tb) << 3) + e5;
                }
                if (rb[q] <= 64u) {
                    seg_put(cur, e5, wa, hi[q], lo[q], rb[q]);
                } else {
                    SegPut st{cur, e5, wa};
                    st = seg_put_long<Sym, TAB>(st, symp, q0 + ((uint64_t)q << R2), RL, n, tab, tab_s, nbins, tmask,
                                                LONG ? reinterpret_cast<const uint64_t *>(bookp + cb_cw_offset())
                                                     : nullptr);
                    cur = st.cur;
                    e5 = st.e5;
                    wa = st.wa;
                }
            }
            // the tile's last word, when partial, belongs to its last segment
            sts_if(tid == kEncThreads - 1 && e5, wa, cur);
        }
        mbar_arrive(&T.done[sl]);
        head += Wa;
        if (++s == (uint32_t)NST) {
            s = 0;
            sph ^= 1u;
        }
    }
}

// Decoupled look-back of tile j by one warp, kLbPer * 32 predecessors per
// step: returns the tile's exclusive stream offset and, in *prev (lane 0),
// the last 32 bits of tile j - 1, taken from the aggregate word the first
// window read; publishes the inclusive offset.  Tile j - 1 usually publishes
// last, so one lane waits for it alone before the window is read.
// A tile that has not published after
// spin_limit polls records HUFF_ERR_TIMEOUT and the look-back goes on with
// what it has (the stream is then invalid).  lo: the field's first tile (0
// for a single field); tiles before it count as a prefix of 0.
static __device__ uint64_t seg_lookback(uint64_t *desc, uint32_t *status, uint64_t j, uint64_t L, uint32_t *prev,
                                        uint32_t spin_limit, uint64_t lo) {
    const uint32_t lane = threadIdx.x & 31;
    uint64_t excl = 0;
    int64_t base = (int64_t)j;                 // look at tiles [base - 128, base)
    uint32_t spins = 0, nap = 32;
    uint64_t a1 = 0;                           // the aggregate word of tile j - 1
    if (lane == 0) {
        uint32_t nap1 = 64;
        a1 = ld_relaxed_u64(&desc[2 * (j - 1)]);
        while (!a1 && spins < spin_limit) {
            spins++;
            __nanosleep(nap1);
            nap1 = nap1 < 512 ? 2 * nap1 : 512;
            a1 = ld_relaxed_u64(&desc[2 * (j - 1)]);
        }
    }
    spins = __shfl_sync(0xFFFFFFFFu, spins, 0);
    for (;;) {
        uint64_t v[kLbPer];
        uint32_t pkey = 0xFFFFFFFFu, zkey = 0xFFFFFFFFu;
#pragma unroll
        for (int q = kLbPer - 1; q >= 0; q--) {
            const uint32_t key = kLbPer * lane + q;
            const int64_t idx = base - 1 - (int64_t)key;
            uint64_t agg = 0, pre = kFlagPre;  // before the field's first tile: prefix 0
            if (idx >= (int64_t)lo) ld_desc(&desc[2 * idx], agg, pre);
            if (idx == (int64_t)j - 1) a1 = agg;
            if (pre) {
                pkey = key;
                v[q] = pre & kValMask;
            } else {
                v[q] = agg & kAggLenMask;
                if (!agg) zkey = key;
            }
        }
        uint32_t pnear = pkey, znear = zkey;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            pnear = min(pnear, __shfl_xor_sync(0xFFFFFFFFu, pnear, o));
            znear = min(znear, __shfl_xor_sync(0xFFFFFFFFu, znear, o));
        }
        if (znear < pnear) {                   // a closer tile has not published yet
            if (++spins > spin_limit) {
                if (lane == 0) set_error(status, HUFF_ERR_TIMEOUT);
                break;
            }
            __nanosleep(nap);
            nap = nap < 1024 ? 2 * nap : 1024;
            continue;
        }
        uint64_t part = 0;
#pragma unroll
        for (int q = 0; q < kLbPer; q++)
            if (kLbPer * lane + q <= pnear) part += v[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        excl += part;
        if (pnear != 0xFFFFFFFFu) break;
        base -= kLbPer * 32;
    }
    if (lane == 0) {
        st_relaxed_u64(&desc[2 * j + 1], kFlagPre | (excl + L));
        // a prefix may be seen before its aggregate word: read it again then
        for (uint32_t sp = 0; !a1 && sp < spin_limit; sp++) a1 = ld_relaxed_u64(&desc[2 * (j - 1)]);
        if (!a1) set_error(status, HUFF_ERR_TIMEOUT);
        *prev = (uint32_t)(a1 >> 24);
    }
    return excl;
}

// Helper warp k of kSegHelpers: for tiles k, k + kSegHelpers, ... the
// look-back gives the stream offset; once every merge thread has stored the
// tile's words, they are copied from the ring into the dense stream and the
// offset is added to the tile's chunk offsets; the tile's ring words and slot
// are then freed in tile order (after the previous tile, another warp's).
template <typename Sym, bool BATCH>
__device__ void seg_helper(const EncArgs &a, const EncField &F0, uint32_t *ring, uint32_t total, SegShared &T,
                           uint32_t k, const uint32_t *sfirst) {
    constexpr uint32_t RW = SegGeom<Sym>::RW;
    constexpr uint32_t SUB = seg_sub_syms<Sym>();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t spin = a.spin_limit ? a.spin_limit : kSpinLimit;
    volatile uint32_t *wdone = &T.wdone;
    for (uint32_t t = k;; t += kSegHelpers) {
        const uint32_t sl = t % kSegSlots;
        const uint32_t ph = (t / kSegSlots) & 1;
        if (!mbar_wait_bounded(&T.full[sl], ph)) {
            if (lane == 0) set_error(BATCH ? a.fields[0].status : F0.status, HUFF_ERR_TIMEOUT);
            return;
        }
        const uint32_t g = T.slot[sl].g;
        if (g >= total) return;
        const uint64_t j = T.slot[sl].j;
        const uint32_t L = T.slot[sl].L, base = T.slot[sl].base, Wa = T.slot[sl].pad;
        const uint32_t fld = T.slot[sl].f;
        const EncField &F = BATCH ? a.fields[fld] : F0;
        const uint64_t ntiles = BATCH ? (uint64_t)(sfirst[fld + 1] - sfirst[fld]) : (uint64_t)F.ntiles;
        uint64_t G = 0;
        uint32_t prev = 0;
        if (j > 0) G = seg_lookback(a.desc, F.status, g, L, &prev, spin, (uint64_t)g - j);
        prev = __shfl_sync(0xFFFFFFFFu, prev, 0);
        const bool last = (j == ntiles - 1);
        if (last && lane == 0) {
            F.offs[F.nchunks] = G + L;
            *F.total_bits = G + L;
        }
        if (!mbar_wait_bounded(&T.done[sl], ph)) {
            if (lane == 0) set_error(F.status, HUFF_ERR_TIMEOUT);
            return;
        }
        const uint32_t fmt = F.format;
        const uint32_t wlog = fmt_wlog(fmt);
        const uint32_t perm = wlog == 5 ? 0x3210u : wlog == 4 ? 0x1032u : 0x0123u;
        const uint64_t cap_bytes = F.cap_words << (wlog - 3);
        const uint32_t g31 = (uint32_t)(G & 31);
        const uint64_t w0 = G >> 5;
        const uint64_t end_bit = G + L;
        const uint32_t tail_bits = (uint32_t)(end_bit & 31);
        const uint32_t nw = (uint32_t)((end_bit >> 5) - w0) + ((last && tail_bits) ? 1 : 0);
        const uint32_t tail_mask = (last && tail_bits) ? ~0u << (32 - tail_bits) : ~0u;
        const uint32_t tail_bytes =
            (last && tail_bits) ? (((tail_bits + (1u << wlog) - 1) >> wlog) << (wlog - 3)) : 4u;
        const uint32_t sh = (32 - g31) & 31;
        // stream word i is the funnel shift of words i and i + 1 from rt: the
        // tile's first ring word, or the one before it (unread: stage memory)
        // when the tile starts mid-word; the last read may be the ring's pad
        const uint32_t *rt = ring + (base % RW) - (g31 ? 1 : 0);
        const uint64_t room_bytes = cap_bytes > 4 * w0 ? cap_bytes - 4 * w0 : 0;
        const bool over = wlog == 5
            ? copy_tile_words<false, 0xFFFFFFFFu>(rt, F.out + w0, 0u, sh, g31, prev, nw, last, tail_bits, tail_mask,
                                                  room_bytes, 4u, 0x3210u, lane)
            : copy_tile_words<true, 0xFFFFFFFFu>(rt, F.out + w0, 0u, sh, g31, prev, nw, last, tail_bits, tail_mask,
                                                 room_bytes, tail_bytes, perm, lane);
        if (over) set_error(F.status, HUFF_ERR_CAPACITY);
        // chunk offsets were written relative to the tile
        const int M = F.chunk_log2;
        const uint64_t chunk_mask = (1ull << M) - 1;
        const uint64_t t0 = j * SUB;
        const uint64_t c_first = (t0 + chunk_mask) >> M;
        const uint64_t tend = t0 + SUB < F.n ? t0 + SUB : F.n;
        const uint64_t c_end = (tend + chunk_mask) >> M;
        uint64_t *offs = F.offs;
        // (a batched launch with short chunks in some field writes every
        // field's chunk offsets to global memory)
        if (seg_coff_smem<Sym>(M) && !(BATCH && a.seg_many)) {
            if (c_first + lane < c_end) offs[c_first + lane] = T.coff[sl][lane] + G;
        } else {
            for (uint64_t c = c_first + lane; c < c_end; c += 32) offs[c] += G;
        }
        __syncwarp();
        if (lane == 0) {
            // free in tile order: after the previous tile (another warp's)
            uint32_t spins = 0;
            while (*wdone != t && ++spins < kSpinLimit) __nanosleep(32);
            if (*wdone != t) set_error(F.status, HUFF_ERR_TIMEOUT);
            __threadfence_block();
            *(volatile uint32_t *)&T.ring_tail = base + Wa;
            *wdone = t + 1;
            mbar_arrive(&T.sfree[sl]);
        }
        __syncwarp();
    }
}

// The merge loop of a field with codewords over 23 bits, out of line: its
// registers are allocated apart from the common loop's.  The launch's
// arguments are passed by value, so that the kernel's own copy keeps no
// address (which would move it to local memory for the common loop too).
template <typename Sym, int TAB, int R2, bool MANY, bool BATCH>
__device__ __noinline__ void seg_merge_long(const EncArgs a, uint8_t *stage, uint32_t *ring, const uint32_t *tab,
                                            uint32_t total, SegShared &T, const uint32_t *sfirst) {
    seg_merge<Sym, TAB, R2, MANY, BATCH, true>(a, stage, ring, tab, total, T, sfirst);
}

// LONGI: the long instance inline (the kernel is then allocated for it) or
// out of line.
template <typename Sym, int TAB, int R2, bool BATCH, bool LONGI>
__device__ __forceinline__ void seg_merge_m(bool many, bool lng, const EncArgs &a, uint8_t *stage, uint32_t *ring,
                                            const uint32_t *tab, uint32_t total, SegShared &T,
                                            const uint32_t *sfirst) {
    if (LONGI && lng) {
        if (many) seg_merge<Sym, TAB, R2, true, BATCH, true>(a, stage, ring, tab, total, T, sfirst);
        else seg_merge<Sym, TAB, R2, false, BATCH, true>(a, stage, ring, tab, total, T, sfirst);
    } else if (lng) {
        if (many) seg_merge_long<Sym, TAB, R2, true, BATCH>(a, stage, ring, tab, total, T, sfirst);
        else seg_merge_long<Sym, TAB, R2, false, BATCH>(a, stage, ring, tab, total, T, sfirst);
    } else {
        if (many) seg_merge<Sym, TAB, R2, true, BATCH, false>(a, stage, ring, tab, total, T, sfirst);
        else seg_merge<Sym, TAB, R2, false, BATCH, false>(a, stage, ring, tab, total, T, sfirst);
    }
}

template <typename Sym, int TAB, bool BATCH = false, bool LONGI = false>
__device__ __forceinline__ void seg_merge_r(int r, bool many, bool lng, const EncArgs &a, uint8_t *stage,
                                            uint32_t *ring, const uint32_t *tab, uint32_t total, SegShared &T,
                                            const uint32_t *sfirst = nullptr) {
    if constexpr (sizeof(Sym) == 1) {
        if (r <= 2) seg_merge_m<Sym, TAB, 2, BATCH, LONGI>(many, lng, a, stage, ring, tab, total, T, sfirst);
        else if (r == 3) seg_merge_m<Sym, TAB, 3, BATCH, LONGI>(many, lng, a, stage, ring, tab, total, T, sfirst);
        else seg_merge_m<Sym, TAB, 4, BATCH, LONGI>(many, lng, a, stage, ring, tab, total, T, sfirst);
    } else if constexpr (sizeof(Sym) == 2) {
        if (r <= 2) seg_merge_m<Sym, TAB, 2, BATCH, LONGI>(many, lng, a, stage, ring, tab, total, T, sfirst);
        else seg_merge_m<Sym, TAB, 3, BATCH, LONGI>(many, lng, a, stage, ring, tab, total, T, sfirst);
    } else {
        if (r <= 1) seg_merge_m<Sym, TAB, 1, BATCH, LONGI>(many, lng, a, stage, ring, tab, total, T, sfirst);
        else seg_merge_m<Sym, TAB, 2, BATCH, LONGI>(many, lng, a, stage, ring, tab, total, T, sfirst);
    }
}

// The segment path of a single-field launch (the header already checked).
// LONGOK: codewords over 23 bits take the segment path too (inline).
template <typename Sym, bool GTAB, bool LONGOK>
__device__ __forceinline__ void seg_body(const EncArgs &a, uint8_t *smem, SegShared &T,
                                         const huff_codebook_header *hdr) {
    constexpr int NST = SegGeom<Sym>::NST;
    constexpr uint32_t SUB = seg_sub_syms<Sym>();
    uint8_t *stage = smem;
    uint32_t *ring = reinterpret_cast<uint32_t *>(smem + NST * seg_sub_bytes<Sym>());
    uint32_t *stab = ring + SegGeom<Sym>::RW + kSegRingPad;
    const uint32_t total = (uint32_t)((a.one.n + SUB - 1) / SUB);
    if (threadIdx.x == 0) {
        T.f0 = a.one;
        T.f0.max_len = hdr->max_len;
        T.f0.nsub = 1;
        T.f0.ntiles = total;
        T.f0.tile_base = 0;
        for (int s = 0; s < NST; s++) mbar_init(&T.bars[s], 1);
        for (int b = 0; b < kSegSlots; b++) {
            mbar_init(&T.full[b], 1);
            mbar_init(&T.done[b], kEncThreads);
            mbar_init(&T.sfree[b], 1);
        }
        T.ring_tail = 0;
        T.wdone = 0;
        fence_barrier_init();
    }
    if (!GTAB) {
        const uint64_t *gcw = reinterpret_cast<const uint64_t *>(a.one.book + cb_cw_offset());
        const uint32_t nb = a.one.nbins;
        for (uint32_t i = threadIdx.x; i < a.tslots; i += blockDim.x)
            stab[i] = seg_entry_from_cw(i < nb ? gcw[i] : 0ull);
    }
    __syncthreads();
    if (threadIdx.x >= kEncThreads) {
        seg_helper<Sym, false>(a, T.f0, ring, total, T, (threadIdx.x - kEncThreads) / 32, nullptr);
        return;
    }
    // the rule's word is the 32-bit ring word the runs are merged into, whatever
    // unit the stream is stored in
    int r = a.reduce_log2 >= 0 ? a.reduce_log2 : enc_rule_r(hdr->total_bits, hdr->nsymbols);
    r = r < seg_r_min<Sym>() ? seg_r_min<Sym>() : (r > seg_r_max<Sym>() ? seg_r_max<Sym>() : r);
    const bool many = (1ull << a.one.chunk_log2) < (uint64_t)seg_lane_syms<Sym>();
    const bool lng = LONGOK && hdr->max_len > kSegEntryLen;
    if (GTAB) seg_merge_r<Sym, 2, false, LONGOK>(r, many, lng, a, stage, ring, a.etab, total, T);
    else seg_merge_r<Sym, 0, false, LONGOK>(r, many, lng, a, stage, ring, stab, total, T);
}

// Single-field encode: the segment path when the codebook allows it, else the
// general encoder.  Dynamic shared memory: the larger of the two layouts.
// LONGOK: the segment path also takes codewords over 23 bits (the instance
// batched plans launch per field); without it such fields run the general
// encoder, and the common loop keeps registers the long one would take.
template <typename Sym, bool GTAB, bool LONGOK>
__global__ void __launch_bounds__(kSegThreads, 2) encode_one_kernel(EncArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ EncShared S;
    __shared__ SegShared T;
    const huff_codebook_header *hdr = reinterpret_cast<const huff_codebook_header *>(a.one.book);
    const bool seg = seg_fits<Sym>(hdr->max_len) && (LONGOK || hdr->max_len <= kSegEntryLen) &&
                     hdr->nbins == a.one.nbins && !fmt_chunk_aligned(a.one.format) && (!GTAB || a.etab != nullptr);
    if (seg) seg_body<Sym, GTAB, LONGOK>(a, smem, T, hdr);
    else if (threadIdx.x < kEncCtaThreads) encode_body<Sym, GTAB, false, false>(a, smem, S);
}

// Batched segment form: one persistent launch over the segment tiles of
// every field the planner gave them (first tile ids in a.seg_first, copied to
// shared memory after the stages and the ring); each field's 32-bit entries
// in global memory (EncField::etab); the reduction factor by rule over those
// fields.  A launch with no such tiles returns at once.
template <typename Sym>
__host__ __device__ inline size_t seg_batch_smem_bytes(uint32_t nfields) {
    return seg_smem_bytes<Sym>(1, true) + ((4ull * (nfields + 1) + 127) & ~127ull);
}

template <typename Sym>
__global__ void __launch_bounds__(kSegThreads, 2) encode_seg_batch_kernel(EncArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ SegShared T;
    constexpr int NST = SegGeom<Sym>::NST;
    uint8_t *stage = smem;
    uint32_t *ring = reinterpret_cast<uint32_t *>(smem + NST * seg_sub_bytes<Sym>());
    uint32_t *sfirst = ring + SegGeom<Sym>::RW + kSegRingPad;
    for (uint32_t i = threadIdx.x; i <= a.nfields; i += blockDim.x) sfirst[i] = a.seg_first[i];
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; s++) mbar_init(&T.bars[s], 1);
        for (int b = 0; b < kSegSlots; b++) {
            mbar_init(&T.full[b], 1);
            mbar_init(&T.done[b], kEncThreads);
            mbar_init(&T.sfree[b], 1);
        }
        T.ring_tail = 0;
        T.wdone = 0;
        fence_barrier_init();
    }
    __syncthreads();
    const uint32_t total = sfirst[a.nfields];
    if (total == 0) return;
    if (threadIdx.x >= kEncThreads) {
        seg_helper<Sym, true>(a, T.f0, ring, total, T, (threadIdx.x - kEncThreads) / 32, sfirst);
        return;
    }
    int r = a.conf->seg_r;
    r = r < seg_r_min<Sym>() ? seg_r_min<Sym>() : (r > seg_r_max<Sym>() ? seg_r_max<Sym>() : r);
    seg_merge_r<Sym, 2, true>(r, a.seg_many != 0, a.conf->seg_long != 0, a, stage, ring, nullptr, total, T, sfirst);
}

using EncOneFn = void (*)(EncArgs);
// Instantiated per symbol width in encode_one_u{8,16,32}.cu.
template <typename Sym>
EncOneFn encode_one_kernel_get(bool gtab, bool long_ok);

}  // namespace huff
