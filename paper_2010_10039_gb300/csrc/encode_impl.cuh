// Encoding (Sec. IV-C) fused with the gathering of Table I ("get blockwise
// code len" prefix sum and "coalescing copy") into one persistent kernel.
//
// Paper design (V100): a chunk of N = 2^M symbols is reduce-merged (each
// thread concatenates 2^r codewords in a register: Merge((a,l)_{2k},
// (a,l)_{2k+1}) = (a_{2k} (+) a_{2k+1}, l_{2k} + l_{2k+1})) and then
// shuffle-merged in shared memory for s = M - r log steps until the chunk is
// one dense run of words; a prefix sum over chunk lengths and a copy then
// gather the chunks into one stream.
//
// GB300 form (this file):
//  * sub-tiles of 4096 (u16) symbols are fetched by the bulk-copy engine into
//    a ring of shared-memory stages (cp.async.bulk + mbarrier); tile ids come
//    from an atomic counter, so tiles start in stream order;
//  * reduce-merge: each thread looks up 2^r codewords in a shared-memory
//    codebook and concatenates them in a 64-bit register; r follows the
//    paper's rule from the average codeword length;
//  * the s log steps of shuffle-merge become one exclusive scan of the merged
//    lengths (a warp scan plus a block-level sum of 8 warp totals), after
//    which every merged run is placed once into a shared-memory bit ring: one
//    data movement instead of s;
//  * the tile's stream offset comes from a decoupled look-back (Merrill &
//    Garland) run by a dedicated warp while the merge warps go on; every tile
//    publishes its length together with its last 32 bits, so a tile writes the
//    word it shares with its predecessor whole: the dense stream is written
//    once, with coalesced plain stores by a dedicated write-out warp, no
//    pre-zeroing and no global atomics, bit-identical to serial packing.
//
// The same kernel encodes a batch of fields in one launch: global tile ids
// run over the fields one after another, every CTA maps the tile it takes to
// its field (binary search in a shared-memory copy of the fields' first tile
// ids), reloads the shared-memory codebook when the field changes, and the
// look-back stops at the field's first tile, so fields share the persistent
// grid but not their streams.
#pragma once

#include "kernels.cuh"

namespace huff {

constexpr int kEncThreads = 256;           // merge threads (8 warps)
constexpr int kEncRPT = 2;                 // consecutive 16-byte vectors per merge thread per sub-tile
constexpr int kEncStages = 4;              // sub-tile stages in flight
constexpr int kEncVecBytes = 16;
constexpr int kEncSubBytes = kEncThreads * kEncRPT * kEncVecBytes;   // 8 KB per sub-tile
constexpr int kEncMaxSubs = 8;             // sub-tiles per tile (fewer when codewords are long)
constexpr int kEncMaxLen = 48;             // longest codeword the bit ring is sized for
constexpr int kSlots = 4;                  // tiles between merge and write-out
constexpr uint32_t kEncSmemTableBins = 4096;
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPre = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr uint64_t kAggLenMask = (1ull << 24) - 1;
constexpr uint32_t kBad32 = 1u << 5;       // flag of a position without codeword (bit 5 is free in u32 entries)
constexpr int kEncCtaThreads = kEncThreads + 64;   // merge warps + look-back warp + write-out warp

struct EncArgs {
    EncField one;                 // single-field launch
    const EncField *fields;       // batched launch: nfields records (device memory)
    const EncBatchConf *conf;     // batched launch
    uint32_t nfields;
    uint32_t tslots;              // shared-memory codebook slots: a power of two >= every nbins
    uint32_t *tile_counter;
    uint64_t *desc;               // look-back descriptors by global tile id, zeroed before the launch
    int32_t reduce_log2;          // single launch: r, or -1 for the average-length rule
    uint32_t nsub_cap;            // at most this many sub-tiles per tile
    const uint32_t *etab;         // single launch, codebook not in shared memory: the codebook's
                                  // 32-bit entries in global memory (used when max_len <= 23)
    uint32_t id_offset;           // added to every tile id taken (0; the failure-detection test
                                  // passes 1, so tile 0 is never encoded)
    uint32_t spin_limit;          // look-back polls before giving up (0: kSpinLimit)
    const uint32_t *seg_first;    // batched segment form: first segment tile of every field, and the
                                  // total after the last (nfields + 1 entries, from the planner)
    uint32_t seg_many;            // batched segment form: some field has chunks shorter than a segment
};

// Tile id taken from the launch's counter.
__device__ __forceinline__ uint32_t take_tile(const EncArgs &a) { return atomicAdd(a.tile_counter, 1u) + a.id_offset; }

template <typename Sym>
struct VecOf {
    static constexpr int N = kEncVecBytes / sizeof(Sym);   // symbols per 16-byte vector
};

template <typename Sym>
__host__ __device__ constexpr uint32_t enc_sub_syms() { return kEncThreads * kEncRPT * VecOf<Sym>::N; }

// Ring of merged bits: 64 KB for u8 sub-tiles (8192 symbols), 32 KB otherwise;
// always large enough for one sub-tile of kEncMaxLen-bit codewords.
template <typename Sym>
__host__ __device__ constexpr uint32_t ring_words() { return sizeof(Sym) == 1 ? 16384u : 8192u; }

// sub-tiles per tile: the tile's worst case (every codeword max_len bits)
// must fit the ring on its own
template <typename Sym>
__host__ __device__ inline uint32_t enc_subs_per_tile(uint32_t max_len, uint32_t cap = kEncMaxSubs) {
    uint32_t m = max_len ? max_len : 1;
    uint32_t k = (ring_words<Sym>() - 64) * 32u / (enc_sub_syms<Sym>() * m);
    if (cap < 1) cap = 1;
    if (cap > (uint32_t)kEncMaxSubs) cap = kEncMaxSubs;
    return k < 1 ? 1 : (k > cap ? cap : k);
}

__device__ __forceinline__ void sym_from_vec(const uint4 &v, uint32_t *s, uint8_t) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 16; j++) s[j] = (w[j >> 2] >> (8 * (j & 3))) & 0xFFu;
}
__device__ __forceinline__ void sym_from_vec(const uint4 &v, uint32_t *s, uint16_t) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 8; j++) s[j] = (j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xFFFFu);
}
__device__ __forceinline__ void sym_from_vec(const uint4 &v, uint32_t *s, uint32_t) {
    s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
}

// ---------------------------------------------------------------- codebook entries
// u32 form (codewords up to 23 bits): the code left-aligned in the top l bits
// and the length l in bits 0..4, e = code << (32 - l) | l; kBad32 for no
// codeword, 0 for padding.  A funnel shift uses only the low 5 bits of its
// shift operand, so funnelshift_l(e, lo, e) = (lo << l) | code appends the
// codeword to a word in one instruction, funnelshift_l(lo, hi, e) carries into
// the high word, and a sum of entries keeps the sum of lengths in bits 0..8
// (codes start at bit 9 or higher).
// u64 form: the codebook's cw (len << 58 | code), 0 for no codeword.

template <typename Entry>
__device__ __forceinline__ Entry entry_from_cw(uint64_t c);
template <>
__device__ __forceinline__ uint32_t entry_from_cw<uint32_t>(uint64_t c) {
    const uint32_t l = (uint32_t)(c >> HUFF_CW_LEN_SHIFT);
    return l ? (((uint32_t)c << (32 - l)) | l) : kBad32;
}
template <>
__device__ __forceinline__ uint64_t entry_from_cw<uint64_t>(uint64_t c) { return c; }

template <typename Entry>
__device__ __forceinline__ uint32_t ent_len(Entry e);
template <>
__device__ __forceinline__ uint32_t ent_len<uint32_t>(uint32_t e) { return e & 31u; }
template <>
__device__ __forceinline__ uint32_t ent_len<uint64_t>(uint64_t e) { return (uint32_t)(e >> HUFF_CW_LEN_SHIFT); }

template <typename Entry>
__device__ __forceinline__ uint64_t ent_code(Entry e);
template <>
__device__ __forceinline__ uint64_t ent_code<uint32_t>(uint32_t e) {
    const uint32_t l = e & 31u;
    return l ? (e >> (32 - l)) : 0u;
}
template <>
__device__ __forceinline__ uint64_t ent_code<uint64_t>(uint64_t e) { return e & ((1ull << HUFF_CW_LEN_SHIFT) - 1); }

// Entry of symbol s.  The shared-memory table has a power-of-two number of
// slots (tmask + 1 >= nbins, slots past nbins have no codeword) and is indexed
// with s & tmask; a symbol beyond the table is caught by the vector range test.
// The global table (large alphabets) is read only for s < nbins.
template <typename Entry, int TAB>
__device__ __forceinline__ Entry table_get(const Entry *tab, const uint64_t *gcw, uint32_t s, uint32_t nbins,
                                           uint32_t tmask) {
    if (TAB == 2) {
        // the entries, precomputed in global memory
        return s < nbins ? __ldg(tab + s) : entry_from_cw<Entry>(0ull);
    } else if (TAB == 1) {
        // converted from the codeword in global memory
        uint64_t c = s < nbins ? __ldg(gcw + s) : 0ull;
        return entry_from_cw<Entry>(c);
    } else {
        return tab[s & tmask];
    }
}

// True when some symbol of the vector is beyond a table of tmask + 1 slots.
__device__ __forceinline__ bool vec_out_of_table(const uint4 &v, uint32_t tmask, uint8_t) {
    const uint32_t m = tmask * 0x01010101u;
    return ((v.x | v.y | v.z | v.w) & ~m) != 0;
}
__device__ __forceinline__ bool vec_out_of_table(const uint4 &v, uint32_t tmask, uint16_t) {
    const uint32_t m = tmask | (tmask << 16);
    return ((v.x | v.y | v.z | v.w) & ~m) != 0;
}
__device__ __forceinline__ bool vec_out_of_table(const uint4 &v, uint32_t tmask, uint32_t) {
    return ((v.x | v.y | v.z | v.w) & ~tmask) != 0;
}

// acc = acc (+) codeword of a u64 entry: append l bits (one step of reduce-merge).
__device__ __forceinline__ void concat64(uint64_t &acc, uint64_t e, uint32_t l) {
    acc = (acc << l) | ent_code<uint64_t>(e);
}

// ---------------------------------------------------------------- bit ring

// Appends codewords one by one (runs longer than 64 bits); completed words go
// to the ring at word base + (bit position >> 5).
template <uint32_t RMASK>
struct BitSink {
    uint64_t acc;
    uint32_t nacc;     // valid low bits of acc (current word so far)
    uint32_t wi;       // word index being filled (not yet masked)
    uint32_t lead;     // placeholder bits of earlier runs in the first word
    uint32_t *buf;

    __device__ __forceinline__ void begin(uint32_t *b, uint32_t base, uint32_t pos) {
        buf = b; wi = base + (pos >> 5); nacc = pos & 31; lead = nacc; acc = 0;
    }
    __device__ __forceinline__ void put(uint32_t c, uint32_t l) {
        acc = (acc << l) | c;
        nacc += l;
        if (nacc >= 32) {
            nacc -= 32;
            uint32_t w = (uint32_t)(acc >> nacc);
            if (lead) atomicOr(&buf[wi & RMASK], w); else buf[wi & RMASK] = w;
            lead = 0;
            wi++;
        }
    }
    __device__ __forceinline__ void put64(uint64_t c, uint32_t l) {
        if (l > 32) { put((uint32_t)(c >> 32), l - 32); put((uint32_t)c, 32); }
        else put((uint32_t)c, l);
    }
    __device__ __forceinline__ void end() {
        if (nacc > lead) atomicOr(&buf[wi & RMASK], (uint32_t)(acc << (32 - nacc)));
    }
};

// Places a merged run of rb (1..64) bits, right-aligned in acc, at tile bit
// pos of a tile that starts at ring word base: at most three words, combined
// with shared-memory OR (the first and last are shared with neighbouring runs).
template <uint32_t RMASK>
__device__ __forceinline__ void place_run(uint32_t *ring, uint32_t base, uint32_t pos, uint64_t acc, uint32_t rb) {
    const uint32_t lo = (uint32_t)acc, hi = (uint32_t)(acc >> 32);
    // MSB-align the run in (ah:al)
    const uint32_t u = 64 - rb;                          // 0..63
    const uint32_t ah = u < 32 ? __funnelshift_l(lo, hi, u) : lo << (u - 32);
    const uint32_t al = u < 32 ? lo << u : 0u;
    // shift right by the bit offset inside the first word: three frame words
    const uint32_t sh = pos & 31, w = base + (pos >> 5);
    const uint32_t f0 = ah >> sh;
    const uint32_t f1 = __funnelshift_r(al, ah, sh);
    const uint32_t f2 = __funnelshift_r(0u, al, sh);
    if (f0) atomicOr(&ring[w & RMASK], f0);
    if (f1) atomicOr(&ring[(w + 1) & RMASK], f1);
    if (f2) atomicOr(&ring[(w + 2) & RMASK], f2);
}

// ---------------------------------------------------------------- look-back descriptors
// 16 bytes per tile, zeroed before the launch:
//   agg = kFlagAgg | last32 << 24 | L    the tile's length and last 32 stream bits
//   pre = kFlagPre | (offset + L)        its inclusive stream offset
// Each word carries everything a reader needs from it, so both are written
// and read with plain (relaxed) 64-bit accesses and no fences.

__device__ __forceinline__ void ld_desc(const uint64_t *d, uint64_t &agg, uint64_t &pre) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(agg), "=l"(pre) : "l"(d) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Decoupled look-back by one warp, 128 predecessor descriptors per step:
// returns the exclusive stream offset of tile j (length L) of a field whose
// descriptors start at desc and, in lane 0, the previous tile's last 32 bits;
// publishes tile j's inclusive offset.  A tile that has not published after
// spin_limit polls records HUFF_ERR_TIMEOUT and the look-back goes on with
// what it has (the stream is then invalid, but the launch completes).
static __device__ uint64_t lookback_warp(uint64_t *desc, uint32_t *status, uint64_t j, uint64_t L, uint32_t *prev_tail,
                                         uint32_t spin_limit) {
    const uint32_t lane = threadIdx.x & 31;
    uint64_t excl = 0;
    int64_t base = (int64_t)j;                 // look at tiles [base-128, base)
    uint32_t spins = 0, nap = 32;
    for (;;) {
        uint64_t v[4];
        uint32_t pkey = 0xFFFFFFFFu, zkey = 0xFFFFFFFFu;
#pragma unroll
        for (int q = 3; q >= 0; q--) {
            const int64_t idx = base - 1 - (int64_t)(4 * lane + q);
            uint64_t agg = 0, pre = kFlagPre;       // before tile 0: prefix 0
            if (idx >= 0) ld_desc(&desc[2 * idx], agg, pre);
            if (pre) { pkey = 4 * lane + q; v[q] = pre & kValMask; }
            else { v[q] = agg & kAggLenMask; if (!agg) zkey = 4 * lane + q; }
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
            __nanosleep(nap);                  // back off: polling competes with the merge warps
            nap = nap < 1024 ? 2 * nap : 1024;
            continue;
        }
        uint64_t part = 0;
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (4 * lane + q <= pnear) part += v[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        excl += part;
        if (pnear != 0xFFFFFFFFu) break;
        base -= 128;
    }
    if (lane == 0) {
        st_relaxed_u64(&desc[2 * j + 1], kFlagPre | (excl + L));
        // the previous tile's last 32 bits travel in its aggregate word
        uint64_t agg = 0;
        for (uint32_t sp = 0; sp < spin_limit; sp++) {
            agg = ld_relaxed_u64(&desc[2 * (j - 1)]);
            if (agg) break;
        }
        if (!agg) set_error(status, HUFF_ERR_TIMEOUT);
        *prev_tail = (uint32_t)(agg >> 24);
    }
    return excl;
}

// ---------------------------------------------------------------- input ring

// Last field whose first tile id is <= g (fields without tiles share the
// first tile id of their successor, so the answer always has tiles).
__device__ __forceinline__ uint32_t field_of(const uint32_t *tbase, uint32_t nfields, uint32_t g) {
    uint32_t lo = 0, hi = nfields;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (tbase[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// Producer of the bulk-copy ring (merge thread 0 only).  Sub-tiles are fetched
// in stream order; a new tile id is taken once every sub-tile of the current
// tile is under way.
struct Producer {
    uint32_t tile;      // global id of the tile being fetched
    uint32_t next;      // id of the tile after it (taken one tile ahead, so its latency is hidden)
    uint32_t sub;       // next sub-tile of it to fetch
    uint32_t slot;      // next ring slot
    uint32_t f;         // field of the tile
    uint32_t nsub;
    uint32_t aligned;
    uint64_t t0;        // first symbol of the tile within its field
    uint64_t n;
    const uint8_t *sym;
};

template <typename Sym, bool BATCH>
__device__ __forceinline__ void produce_next(const EncArgs &a, const EncField *fields, const uint32_t *tbase,
                                             Producer &p, uint32_t total, uint8_t *stage, uint64_t *bars,
                                             volatile uint32_t *s_stage_tile, volatile uint32_t *s_stage_field) {
    constexpr uint32_t SUB = enc_sub_syms<Sym>();
    if (p.sub >= p.nsub && p.tile < total) {
        p.tile = p.next;
        if (p.tile < total) p.next = take_tile(a);   // predicated: not waited on here
        p.sub = 0;
        if (p.tile < total) {
            p.f = BATCH ? field_of(tbase, a.nfields, p.tile) : 0u;
            const EncField &F = fields[p.f];
            p.nsub = F.nsub;
            p.n = F.n;
            p.sym = F.sym;
            p.aligned = F.aligned;
            p.t0 = (uint64_t)(p.tile - F.tile_base) * (SUB * p.nsub);
        }
    }
    const int s = (int)(p.slot % kEncStages);
    s_stage_tile[s] = p.tile;
    s_stage_field[s] = p.f;
    if (p.tile < total) {
        const uint64_t s0 = p.t0 + (uint64_t)p.sub * SUB;
        if (p.aligned && s0 + SUB <= p.n) {
            mbar_arrive_expect_tx(&bars[s], kEncSubBytes);
            bulk_g2s(stage + s * kEncSubBytes, p.sym + s0 * sizeof(Sym), kEncSubBytes, &bars[s]);
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars[s])) : "memory");
        }
    }
    p.sub++;
    p.slot++;
}

// Producer of a single-field launch: the field is the kernel parameter, so
// only the position lives in (thread 0's) registers.
struct ProducerOne {
    uint32_t tile;
    uint32_t next;
    uint32_t sub;
    uint32_t slot;
};

template <typename Sym>
__device__ __forceinline__ void produce_next_one(const EncArgs &a, ProducerOne &p, uint32_t nsub, uint32_t total,
                                                 uint8_t *stage, uint64_t *bars, volatile uint32_t *s_stage_tile) {
    constexpr uint32_t SUB = enc_sub_syms<Sym>();
    if (p.sub >= nsub && p.tile < total) {
        p.tile = p.next;
        // predicated, not selected: nothing reads the new id before the next
        // tile switch, so the atomic's round trip does not stall the warp
        if (p.tile < total) p.next = take_tile(a);
        p.sub = 0;
    }
    const int s = (int)(p.slot % kEncStages);
    s_stage_tile[s] = p.tile;
    if (p.tile < total) {
        const uint64_t s0 = ((uint64_t)p.tile * nsub + p.sub) * SUB;
        if (a.one.aligned && s0 + SUB <= a.one.n) {
            mbar_arrive_expect_tx(&bars[s], kEncSubBytes);
            bulk_g2s(stage + s * kEncSubBytes, a.one.sym + s0 * sizeof(Sym), kEncSubBytes, &bars[s]);
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars[s])) : "memory");
        }
    }
    p.sub++;
    p.slot++;
}

__device__ __forceinline__ void merge_sync() {       // the 8 merge warps only
    asm volatile("bar.sync 1, %0;" ::"n"(kEncThreads) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// A tile between merge and write-out.
struct TileSlot {
    uint64_t j;           // tile index within its field
    uint64_t G;           // exclusive stream offset
    uint32_t g;           // global tile id (>= the launch's total: no more tiles)
    uint32_t f;           // field
    uint32_t L;           // length in bits
    uint32_t base;        // first ring word (running counter, masked on use)
    uint32_t prev;        // last 32 bits of the tile before it
    uint32_t pad;
};

struct EncShared {
    uint64_t bars[kEncStages];      // sub-tile stages (bulk copies)
    uint64_t full[kSlots];          // merge -> look-back: tile merged and its aggregate published
    uint64_t gready[kSlots];        // look-back -> write-out: offset known
    uint64_t sfree[kSlots];         // write-out -> merge: slot reusable
    uint32_t stage_tile[kEncStages];
    uint32_t stage_field[kEncStages];
    TileSlot slot[kSlots];
    uint32_t ring_tail;             // ring words before this counter are free again
    uint32_t wsum[2][kEncThreads / 32];   // warp totals of the merged lengths (double-buffered)
    EncField f0;                    // the field of a single-field launch, completed from its codebook
    EncField mf;                    // the field the merge warps are in
    Producer prod;                  // bulk-copy producer state (merge thread 0)
};

// ---------------------------------------------------------------- merge warps

// Reduce-merge of one 16-byte vector: 2^R2 codewords per run, concatenated
// in a 64-bit register.  FULL: all symbols valid and below nbins.  `bad`
// collects kBad32 when a valid position has no codeword.
template <typename Sym, typename Entry, int TAB, int R2, bool FULL>
__device__ __forceinline__ uint32_t merge_vec(const uint32_t *sv, uint32_t valid, const Entry *tab,
                                              const uint64_t *gcw, uint32_t nbins, uint32_t tmask, uint64_t *acc,
                                              uint32_t *rb, uint32_t &bad) {
    constexpr int V = VecOf<Sym>::N;
    constexpr int RL = 1 << R2;
    constexpr int NR = V / RL;
    uint32_t tot = 0;
#pragma unroll
    for (int r = 0; r < NR; r++) {
        if constexpr (sizeof(Entry) == 4) {
            // lo/hi: the run so far; esum: sum of entries (lengths in bits 0..8)
            uint32_t lo = 0, hi = 0, esum = 0;
#pragma unroll
            for (int x = 0; x < RL; x++) {
                const int xi = r * RL + x;
                uint32_t en = (uint32_t)table_get<Entry, TAB>(tab, gcw, sv[xi], nbins, tmask);
                if (!FULL && xi >= (int)valid) en = 0u;               // padding past n: length 0
                bad |= en;
                hi = __funnelshift_l(lo, hi, en);
                lo = __funnelshift_l(en, lo, en);
                esum += en;
            }
            acc[r] = ((uint64_t)hi << 32) | lo;
            rb[r] = esum & 511u;
        } else {
            uint64_t ac = 0;
            uint32_t bb = 0;
#pragma unroll
            for (int x = 0; x < RL; x++) {
                const int xi = r * RL + x;
                Entry en = table_get<Entry, TAB>(tab, gcw, sv[xi], nbins, tmask);
                if (!FULL && xi >= (int)valid) en = (Entry)0;        // padding past n: length 0
                else bad |= en == 0 ? kBad32 : 0u;
                const uint32_t l = ent_len<Entry>(en);
                concat64(ac, en, l);
                bb += l;
            }
            acc[r] = ac;
            rb[r] = bb;
        }
        tot += rb[r];
    }
    return tot;
}

// Places a run longer than 64 bits codeword by codeword (symbols from global
// memory: the stage may be refilled already).  Kept out of line so the rare
// path adds no registers or instructions to the placement loop.
template <typename Sym, typename Entry, int TAB, uint32_t RMASK>
__device__ __noinline__ void place_long_run(uint32_t *ring, uint32_t base, uint32_t pos, const Sym *symp,
                                            uint64_t first, int count, uint64_t n, const Entry *tab,
                                            const uint64_t *gcw, uint32_t nbins, uint32_t tmask) {
    BitSink<RMASK> sink;
    sink.begin(ring, base, pos);
    for (int x = 0; x < count; x++) {
        const uint64_t i = first + x;
        if (i >= n) break;
        Entry en = table_get<Entry, TAB>(tab, gcw, (uint32_t)symp[i], nbins, tmask);
        const uint32_t l = ent_len<Entry>(en);
        if (l) sink.put64(ent_code<Entry>(en), l);
    }
    sink.end();
}

// Loads the shared-memory codebook of a field: tslots entries, those past
// nbins without codeword.  Merge threads only.
template <typename Entry>
__device__ __forceinline__ void load_table(Entry *tab, uint32_t tslots, const EncField &F) {
    const uint64_t *gcw = reinterpret_cast<const uint64_t *>(F.book + cb_cw_offset());
    const uint32_t nb = F.nbins;
    for (uint32_t i = threadIdx.x; i < tslots; i += kEncThreads)
        tab[i] = entry_from_cw<Entry>(i < nb ? gcw[i] : 0ull);
}

// The 8 merge warps: reduce-merge every tile into the bit ring, publish its
// aggregate and hand it to the look-back and write-out warps.  R2 = r:
// 2^r codewords per register.
template <typename Sym, typename Entry, int TAB, int R2, bool BATCH, bool CALIGN>
__device__ void merge_warps(const EncArgs &a, const EncField *fields, const uint32_t *tbase, uint8_t *stage,
                            uint32_t *ring, Entry *tab, uint32_t total, uint32_t nsub1, uint32_t max_len1,
                            EncShared &S) {
    constexpr int V = VecOf<Sym>::N;              // symbols per 16-byte vector
    constexpr int RL = 1 << R2;                   // symbols per merged run
    constexpr int NR = V / RL;                    // runs per vector
    static_assert(RL <= V, "a run stays inside one vector");
    constexpr uint32_t SUB = enc_sub_syms<Sym>();
    constexpr uint32_t RW = ring_words<Sym>();
    constexpr uint32_t RMASK = RW - 1;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t tmask = a.tslots - 1;
    volatile uint32_t *stage_tile = S.stage_tile;
    volatile uint32_t *stage_field = S.stage_field;
    volatile uint32_t *ring_tail = &S.ring_tail;

    // A batch producer keeps its state in shared memory (only thread 0 touches
    // it, and it would otherwise hold registers in every merge thread); a
    // single-field producer needs four registers.
    Producer &prod = S.prod;
    ProducerOne one{0u, 0u, nsub1, 0u};
    if (tid == 0) {
        if (BATCH) {
            prod.slot = 0;
            prod.sub = 0;
            prod.nsub = 0;
            prod.tile = 0;
            prod.f = 0;
            prod.next = take_tile(a);
        } else {
            one.next = take_tile(a);
            for (int i = 0; i < kEncStages; i++) stage_field[i] = 0;
        }
        for (int i = 0; i < kEncStages; i++) {
            if (BATCH) produce_next<Sym, true>(a, fields, tbase, prod, total, stage, S.bars, stage_tile, stage_field);
            else produce_next_one<Sym>(a, one, nsub1, total, stage, S.bars, stage_tile);
        }
    }
    merge_sync();

    uint32_t it = 0, t = 0, base = 0, cur_f = 0xFFFFFFFFu;
    // chunk-aligned layout (CALIGN: single-field launches only): a chunk is a
    // group of pad_group = 2^M / (warp's symbols) consecutive merge warps,
    // 1..8 (checked on the host)
    constexpr uint32_t kWarpLog2 = 5 + 1 + (sizeof(Sym) == 1 ? 4 : sizeof(Sym) == 2 ? 3 : 2);
    static_assert((1u << kWarpLog2) == 32u * kEncRPT * VecOf<Sym>::N, "warp symbols");
    static_assert(!(CALIGN && BATCH), "the batched form writes the dense layout");
    const uint32_t pad_group = CALIGN ? 1u << (a.one.chunk_log2 - kWarpLog2) : 1u;
    const uint32_t pad_mask = (1u << fmt_wlog(a.one.format)) - 1;
    for (;; t++) {
        const uint32_t g = stage_tile[it % kEncStages];
        const uint32_t f = stage_field[it % kEncStages];
        const uint32_t sl = t % kSlots;
        if (t >= kSlots && !mbar_wait_bounded(&S.sfree[sl], ((t / kSlots) - 1) & 1))
            set_error(fields[f].status, HUFF_ERR_TIMEOUT);
        if (g >= total) {
            if (tid == 0) {
                S.slot[sl].g = 0xFFFFFFFFu;
                mbar_arrive(&S.full[sl]);
            }
            break;
        }
        if (f != cur_f) {
            // every merge thread is past its last lookup in the previous field's table
            if (TAB == 0) load_table<Entry>(tab, a.tslots, BATCH ? fields[f] : a.one);
            if (BATCH && tid == 0) S.mf = fields[f];
            cur_f = f;
            merge_sync();
        }
        // A batch reads the field's values from shared memory where they are
        // used, so they hold no registers across the merge loop; a single-field
        // launch reads them from the kernel parameters.
        const EncField &F = BATCH ? S.mf : a.one;
        const uint32_t nsub = BATCH ? S.mf.nsub : nsub1;
        const uint64_t j = BATCH ? g - S.mf.tile_base : g;
        const uint64_t t0 = j * (uint64_t)(SUB * nsub);
        uint32_t running = 0;

        for (uint32_t sub = 0; sub < nsub; sub++, it++) {
            const uint64_t n = F.n;
            const uint32_t nbins = F.nbins;
            const Sym *symp = reinterpret_cast<const Sym *>(F.sym);
            const uint64_t *gcw = reinterpret_cast<const uint64_t *>(F.book + cb_cw_offset());
            uint32_t *status = F.status;
            const int s = (int)(it % kEncStages);
            const uint32_t parity = (it / kEncStages) & 1;
            const uint64_t s0 = t0 + (uint64_t)sub * SUB;
            const bool full = F.aligned && s0 + SUB <= n;
            if (tid == 0) {
                // room in the ring for this sub-tile's worst case
                const uint32_t sub_words = (SUB * (BATCH ? S.mf.max_len : max_len1) + 31) / 32 + 2;
                const uint32_t need_end = base + running / 32 + sub_words;
                uint32_t spins = 0;
                while (need_end - *ring_tail > RW) {
                    if (++spins > kSpinLimit) { set_error(status, HUFF_ERR_TIMEOUT); break; }
                    __nanosleep(32);
                }
                __threadfence_block();
            }
            if (!mbar_wait_bounded(&S.bars[s], parity)) set_error(status, HUFF_ERR_TIMEOUT);
            const uint8_t *st = stage + s * kEncSubBytes;

            // ---- reduce-merge: look up 2^r codewords and concatenate them in a register
            uint64_t acc[kEncRPT][NR];
            uint32_t rb[kEncRPT][NR];
            uint32_t bits[kEncRPT];
            uint32_t bad = 0;
#pragma unroll
            for (int k = 0; k < kEncRPT; k++) {
                const uint32_t q = kEncRPT * tid + k;          // this thread's vectors are consecutive
                uint32_t sv[V];
                if (full) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(st + q * kEncVecBytes);
                    sym_from_vec(v, sv, Sym());
                    if (TAB == 0 && vec_out_of_table(v, tmask, Sym())) bad |= kBad32;
                    bits[k] = merge_vec<Sym, Entry, TAB, R2, true>(sv, V, tab, gcw, nbins, tmask, acc[k], rb[k], bad);
                } else {
                    const uint64_t i0 = s0 + (uint64_t)q * V;
                    const uint32_t vl = i0 >= n ? 0 : (n - i0 < V ? (uint32_t)(n - i0) : V);
#pragma unroll
                    for (int x = 0; x < V; x++) sv[x] = x < (int)vl ? (uint32_t)symp[i0 + x] : 0u;
#pragma unroll
                    for (int x = 0; x < V; x++)
                        if (x < (int)vl && sv[x] > tmask) bad |= kBad32;
                    bits[k] = merge_vec<Sym, Entry, TAB, R2, false>(sv, vl, tab, gcw, nbins, tmask, acc[k], rb[k], bad);
                }
            }
            if (bad & kBad32) {
                // a symbol without codeword, or out of range: find out which
                uint32_t code = HUFF_ERR_NOT_IN_CODEBOOK;
#pragma unroll
                for (int k = 0; k < kEncRPT; k++) {
                    const uint32_t q = kEncRPT * tid + k;
                    for (int x = 0; x < V; x++) {
                        const uint64_t i = s0 + (uint64_t)q * V + x;
                        if (i < n) {
                            uint32_t sx = full ? (uint32_t)reinterpret_cast<const Sym *>(st + q * kEncVecBytes)[x]
                                               : (uint32_t)symp[i];
                            if (sx >= nbins) code = HUFF_ERR_SYMBOL_RANGE;
                        }
                    }
                }
                set_error(status, code);
            }

            // ---- shuffle-merge as one scan: bit offset of this thread's runs in the tile
            const uint32_t mine = bits[0] + bits[1];
            uint32_t inc = mine;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= o) inc += y;
            }
            uint32_t *ws = S.wsum[it & 1];
            if (lane == 31) ws[warp] = inc;
            merge_sync();
            // every merge thread has read stage s: refill it
            if (tid == 0) {
                if (BATCH) produce_next<Sym, true>(a, fields, tbase, prod, total, stage, S.bars, stage_tile, stage_field);
                else produce_next_one<Sym>(a, one, nsub1, total, stage, S.bars, stage_tile);
            }
            // exclusive prefix of the 8 warp totals, by shuffles
            constexpr int NW = kEncThreads / 32;
            uint32_t wt = lane < NW ? ws[lane] : 0u;
            if constexpr (CALIGN) {
                // the last warp of each chunk carries the padding up to the
                // next unit boundary; sub-tiles start at unit boundaries, so
                // the padding depends only on the chunk's own length
                uint32_t gs = wt;
                for (uint32_t o = 1; o < pad_group; o <<= 1) gs += __shfl_xor_sync(0xFFFFFFFFu, gs, o);
                if ((lane & (pad_group - 1)) == pad_group - 1) wt += ((gs + pad_mask) & ~pad_mask) - gs;
            }
            uint32_t wi = wt;
#pragma unroll
            for (int o = 1; o < NW; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (lane >= o) wi += y;
            }
            const uint32_t wbase = __shfl_sync(0xFFFFFFFFu, wi - wt, warp);
            const uint32_t Lsub = __shfl_sync(0xFFFFFFFFu, wi, NW - 1);
            uint32_t pos = running + wbase + inc - mine;

            // ---- place each merged run once; chunk offsets relative to the tile for now
            uint64_t *offs = F.offs;
            const int M = F.chunk_log2;
            const uint64_t chunk_mask = (1ull << M) - 1;
            // chunks of at most a sub-tile start at vectors q with q % vpc == 0 (vpc a power of two)
            const bool small_chunks = (1ull << M) <= SUB;
            const uint32_t vpc = small_chunks ? (uint32_t)((1ull << M) / V) : 1u;
#pragma unroll
            for (int k = 0; k < kEncRPT; k++) {
                const uint32_t q = kEncRPT * tid + k;
                if (small_chunks) {
                    if ((q & (vpc - 1)) == 0 && (full || s0 + (uint64_t)q * V < n)) offs[(s0 + q * V) >> M] = pos;
                } else if (q == 0 && (s0 & chunk_mask) == 0 && s0 < n) {
                    offs[s0 >> M] = pos;
                }
#pragma unroll
                for (int r = 0; r < NR; r++) {
                    const uint32_t bb = rb[k][r];
                    if (bb <= 64) {
                        if (bb) place_run<RMASK>(ring, base, pos, acc[k][r], bb);
                    } else {
                        // longer than the register (rare): codeword by codeword, out of line
                        place_long_run<Sym, Entry, TAB, RMASK>(ring, base, pos, symp,
                                                               s0 + (uint64_t)q * V + r * RL, RL, n, tab, gcw,
                                                               nbins, tmask);
                    }
                    pos += bb;
                }
            }
            running += Lsub;
        }
        merge_sync();                                      // tile bits complete in the ring
        const uint32_t L = running;
        if (tid == 0) {
            // publish the tile's length and last 32 bits; hand it on
            uint32_t last32 = 0;
            if (L >= 32) {
                uint32_t bb = L - 32, w = base + (bb >> 5), sh = bb & 31;
                last32 = sh ? (ring[w & RMASK] << sh) | (ring[(w + 1) & RMASK] >> (32 - sh)) : ring[w & RMASK];
            } else if (L) {
                last32 = ring[base & RMASK] >> (32 - L);
            }
            st_relaxed_u64(&a.desc[2 * (uint64_t)g], kFlagAgg | ((uint64_t)last32 << 24) | L);
            if (j == 0) st_relaxed_u64(&a.desc[2 * (uint64_t)g + 1], kFlagPre | L);
            S.slot[sl].g = g;
            S.slot[sl].f = f;
            S.slot[sl].j = j;
            S.slot[sl].L = L;
            S.slot[sl].base = base;
            mbar_arrive(&S.full[sl]);
        }
        base += (L + 31) / 32;
    }
}

// ---------------------------------------------------------------- look-back warp

// Resolves the stream offset of each merged tile, in order.
static __device__ void lookback_loop(const EncArgs &a, const EncField *fields, uint32_t total, EncShared &S) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t t = 0;; t++) {
        const uint32_t sl = t % kSlots;
        if (!mbar_wait_bounded(&S.full[sl], (t / kSlots) & 1)) {
            if (lane == 0) set_error(fields[0].status, HUFF_ERR_TIMEOUT);
            return;
        }
        const uint32_t g = S.slot[sl].g;
        if (g < total) {
            const EncField &F = fields[S.slot[sl].f];
            const uint64_t j = S.slot[sl].j;
            const uint32_t L = S.slot[sl].L;
            uint64_t G = 0;
            uint32_t prev = 0;
            if (j > 0) G = lookback_warp(a.desc + 2 * (uint64_t)F.tile_base, F.status, j, L, &prev,
                                         a.spin_limit ? a.spin_limit : kSpinLimit);
            if (lane == 0) {
                S.slot[sl].G = G;
                S.slot[sl].prev = prev;
                if (j == F.ntiles - 1) {
                    F.offs[F.nchunks] = fmt_chunk_aligned(F.format) ? (G + L) >> fmt_wlog(F.format) : G + L;
                    *F.total_bits = G + L;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.gready[sl]);
        if (g >= total) return;
    }
}

// ---------------------------------------------------------------- write-out warp

// Copies one tile's nw stream words from the ring to outw (the stream's word
// w0 on): word i is the funnel shift of ring words wb + i and wb + i + 1 (one
// SHF, which also covers sh = 0); the first word, when the tile starts
// mid-word, is completed with the previous tile's last bits.  A block of 128
// words that is whole, inside the capacity, does not hold the shared first
// word and does not hold a masked last word takes no per-word checks (the
// test is warp-uniform).  Four independent words per lane per step, four
// coalesced stores.  TYPED: units of 8 or 16 bits, so each word is permuted
// into stream order (perm) and the capacity and the stream's last word are
// counted in bytes (narrow stores for a last word only partly inside).
// Returns whether a word fell outside the capacity (it is not written).
template <bool TYPED, uint32_t RMASK>
__device__ __forceinline__ bool copy_tile_words(const uint32_t *ring, uint32_t *outw, uint32_t wb, uint32_t sh,
                                                uint32_t g31, uint32_t prev, uint32_t nw, bool last,
                                                uint32_t tail_bits, uint32_t tail_mask, uint64_t room_bytes,
                                                uint32_t tail_bytes, uint32_t perm, uint32_t lane) {
    const uint64_t room = room_bytes >> 2;                                   // whole words
    bool over = false;
    for (uint32_t b0 = 0; b0 < nw; b0 += 128) {
        const bool fast = b0 + 128 <= nw && (uint64_t)(b0 + 128) <= room && !(b0 == 0 && g31) &&
                          !(b0 + 128 == nw && last && tail_bits);
        uint32_t val[4];
        if (fast) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t i = b0 + 32 * k + lane;
                val[k] = __funnelshift_l(ring[(wb + i + 1) & RMASK], ring[(wb + i) & RMASK], sh);
                if (TYPED) val[k] = __byte_perm(val[k], 0u, perm);
            }
#pragma unroll
            for (int k = 0; k < 4; k++) outw[b0 + 32 * k + lane] = val[k];
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t i = b0 + 32 * k + lane;
                const uint32_t hi = ring[(wb + i) & RMASK], lo = ring[(wb + i + 1) & RMASK];
                val[k] = __funnelshift_l(lo, hi, sh);
                if (i == 0 && g31) val[k] = ((prev & ((1u << g31) - 1)) << (32 - g31)) | (lo >> g31);
                if (i == nw - 1) val[k] &= tail_mask;
                if (TYPED) val[k] = __byte_perm(val[k], 0u, perm);
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t i = b0 + 32 * k + lane;
                if (i < nw) {
                    if (!TYPED) {
                        if ((uint64_t)i < room) outw[i] = val[k]; else over = true;
                    } else {
                        const uint32_t want = i == nw - 1 ? tail_bytes : 4u;
                        if (4ull * i + want <= room_bytes) {
                            if (want == 4) {
                                outw[i] = val[k];
                            } else if (want == 2) {
                                reinterpret_cast<uint16_t *>(outw + i)[0] = (uint16_t)val[k];
                            } else {
                                uint8_t *ob = reinterpret_cast<uint8_t *>(outw + i);
                                for (uint32_t x = 0; x < want; x++) ob[x] = (uint8_t)(val[k] >> (8 * x));
                            }
                        } else {
                            over = true;
                        }
                    }
                }
            }
        }
    }
    return over;
}

// Copies each tile from the ring into the dense stream at its offset (the word
// it shares with the previous tile is completed with the previous tile's last
// bits), fixes the tile's chunk offsets and frees its ring words.
template <typename Sym>
__device__ void writeout_loop(const EncField *fields, uint32_t *ring, uint32_t total, EncShared &S) {
    constexpr uint32_t RMASK = ring_words<Sym>() - 1;
    constexpr uint32_t SUB = enc_sub_syms<Sym>();
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t t = 0;; t++) {
        const uint32_t sl = t % kSlots;
        if (!mbar_wait_bounded(&S.gready[sl], (t / kSlots) & 1)) {
            if (lane == 0) set_error(fields[0].status, HUFF_ERR_TIMEOUT);
            return;
        }
        const uint32_t g = S.slot[sl].g;
        if (g >= total) return;
        const EncField &F = fields[S.slot[sl].f];
        const uint64_t j = S.slot[sl].j;
        const uint64_t G = S.slot[sl].G;
        const uint32_t L = S.slot[sl].L, base = S.slot[sl].base, prev = S.slot[sl].prev;
        const bool last = (j == F.ntiles - 1);
        uint32_t *out = F.out;
        // capacity and stream end in bytes: units of W = 2^wlog bits (W < 32
        // stores each 32-bit word's units in stream order: bytes or halves
        // swapped; a last word only partly inside takes narrow stores)
        const uint32_t fmt = F.format;
        const uint32_t wlog = fmt_wlog(fmt);
        const uint32_t perm = wlog == 5 ? 0x3210u : wlog == 4 ? 0x1032u : 0x0123u;
        const uint64_t cap_bytes = F.cap_words << (wlog - 3);
        const uint32_t g31 = (uint32_t)(G & 31);
        const uint64_t w0 = G >> 5;
        const uint64_t end_bit = G + L;
        const uint32_t tail_bits = (uint32_t)(end_bit & 31);
        const uint32_t nw = (uint32_t)((end_bit >> 5) - w0) + ((last && tail_bits) ? 1 : 0);
        // the last tile of a field also writes its partial final word, whose
        // ring neighbour may already hold the next tile (of another field)
        const uint32_t tail_mask = (last && tail_bits) ? ~0u << (32 - tail_bits) : ~0u;
        // bytes of the stream's last word that belong to it (whole units)
        const uint32_t tail_bytes = (last && tail_bits) ? (((tail_bits + (1u << wlog) - 1) >> wlog) << (wlog - 3)) : 4u;
        // stream word w0 + i holds tile bits [32 i - g31, 32 i - g31 + 32), i.e.
        // the funnel shift of ring words wb + i and wb + i + 1
        const uint32_t sh = (32 - g31) & 31;
        const uint32_t wb = base - (g31 ? 1u : 0u);
        const uint64_t room_bytes = cap_bytes > 4 * w0 ? cap_bytes - 4 * w0 : 0;   // bytes writable from w0
        const bool over = wlog == 5
            ? copy_tile_words<false, RMASK>(ring, out + w0, wb, sh, g31, prev, nw, last, tail_bits, tail_mask,
                                            room_bytes, 4u, 0x3210u, lane)
            : copy_tile_words<true, RMASK>(ring, out + w0, wb, sh, g31, prev, nw, last, tail_bits, tail_mask,
                                           room_bytes, tail_bytes, perm, lane);
        if (over) set_error(F.status, HUFF_ERR_CAPACITY);
        // chunk offsets were written relative to the tile
        const int M = F.chunk_log2;
        const uint64_t chunk_mask = (1ull << M) - 1;
        const uint64_t TILE = (uint64_t)SUB * F.nsub;
        const uint64_t t0 = j * TILE;
        const uint64_t c_first = (t0 + chunk_mask) >> M;
        const uint64_t tend = t0 + TILE < F.n ? t0 + TILE : F.n;
        const uint64_t c_end = (tend + chunk_mask) >> M;
        uint64_t *offs = F.offs;
        if (fmt_chunk_aligned(fmt)) {
            for (uint64_t c = c_first + lane; c < c_end; c += 32) offs[c] = (offs[c] + G) >> wlog;
        } else {
            for (uint64_t c = c_first + lane; c < c_end; c += 32) offs[c] += G;
        }
        __syncwarp();
        const uint32_t used = (L + 31) / 32;
        for (uint32_t wz = 0; wz < used; wz += 128) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t w = wz + 32 * k + lane;
                if (w < used) ring[(base + w) & RMASK] = 0;
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            *(volatile uint32_t *)&S.ring_tail = base + used;
            mbar_arrive(&S.sfree[sl]);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- kernel

// Largest and smallest reduction factor per symbol width: a run stays inside
// one 16-byte vector, and at most 4 runs per vector are held in registers.
template <typename Sym>
__host__ __device__ constexpr int enc_r_max() { return sizeof(Sym) == 1 ? 4 : sizeof(Sym) == 2 ? 3 : 2; }
template <typename Sym>
__host__ __device__ constexpr int enc_r_min() { return sizeof(Sym) == 4 ? 0 : 2; }

template <typename Sym>
__host__ __device__ inline int enc_clamp_r(int r) {
    return r < enc_r_min<Sym>() ? enc_r_min<Sym>() : (r > enc_r_max<Sym>() ? enc_r_max<Sym>() : r);
}

// Reduction factor rule of Sec. IV-C: floor(log2 beta) + r + 1 = log2(W)
// (W = 2^wlog), beta = total_bits / nsymbols the average codeword length,
// clamped to [0, wlog] like huff_reduce_factor (the caller then applies the
// register clamp).  The encoders take W = 32, the word their runs are merged
// into, for every stored unit width.
__host__ __device__ inline int enc_rule_r(uint64_t total_bits, uint64_t nsymbols, int wlog = 5) {
    // floor(log2(beta)): largest f with nsymbols * 2^f <= total_bits
    int f = 0;
    while (f < 62 && nsymbols && (nsymbols << (f + 1)) <= total_bits && ((nsymbols << (f + 1)) >> (f + 1)) == nsymbols)
        f++;
    return f > wlog - 1 ? 0 : wlog - 1 - f;
}

template <typename Sym, typename Entry, int TAB, bool BATCH, bool CALIGN>
__device__ void merge_dispatch(int r, const EncArgs &a, const EncField *fields, const uint32_t *tbase,
                               uint8_t *stage, uint32_t *ring, Entry *tab, uint32_t total, uint32_t nsub1,
                               uint32_t max_len1, EncShared &S) {
    switch (r) {
        case 0: if constexpr (VecOf<Sym>::N <= 4) merge_warps<Sym, Entry, TAB, 0, BATCH, CALIGN>(a, fields, tbase, stage, ring, tab, total, nsub1, max_len1, S); break;
        case 1: if constexpr (VecOf<Sym>::N <= 4) merge_warps<Sym, Entry, TAB, 1, BATCH, CALIGN>(a, fields, tbase, stage, ring, tab, total, nsub1, max_len1, S); break;
        case 2: merge_warps<Sym, Entry, TAB, 2, BATCH, CALIGN>(a, fields, tbase, stage, ring, tab, total, nsub1, max_len1, S); break;
        case 3: if constexpr (VecOf<Sym>::N >= 8) merge_warps<Sym, Entry, TAB, 3, BATCH, CALIGN>(a, fields, tbase, stage, ring, tab, total, nsub1, max_len1, S); break;
        default: if constexpr (VecOf<Sym>::N >= 16) merge_warps<Sym, Entry, TAB, 4, BATCH, CALIGN>(a, fields, tbase, stage, ring, tab, total, nsub1, max_len1, S); break;
    }
}

// Shared memory of a launch: stages, bit ring, codebook table (unless read
// from global memory) and, for a batch, the fields' first tile ids.
template <typename Sym>
__host__ __device__ inline size_t enc_smem_bytes(bool gtab, uint32_t tslots, uint32_t nfields_batch) {
    return kEncStages * kEncSubBytes + ring_words<Sym>() * 4 + (gtab ? 0 : tslots * 8ull) +
           (nfields_batch ? 4ull * (nfields_batch + 1) : 0);
}

// The kernel body over the dynamic shared memory smem (stages, bit ring,
// codebook table, batch tile bases) and the launch's EncShared record.
template <typename Sym, bool GTAB, bool BATCH, bool CALIGN>
__device__ __forceinline__ void encode_body(const EncArgs &a, uint8_t *smem, EncShared &S) {
    constexpr uint32_t RW = ring_words<Sym>();
    uint8_t *stage = smem;
    uint32_t *ring = reinterpret_cast<uint32_t *>(smem + kEncStages * kEncSubBytes);
    uint64_t *tab = reinterpret_cast<uint64_t *>(ring + RW);
    uint32_t *tbase = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(tab) + (GTAB ? 0 : a.tslots * 8ull));

    uint32_t total, nsub1 = 0, max_len1 = 0;
    int r;
    bool e32;
    const EncField *fields;
    if (BATCH) {
        const EncBatchConf c = *a.conf;
        total = c.total_tiles;
        r = c.r;
        e32 = c.entry32 != 0;
        fields = a.fields;
        for (uint32_t i = threadIdx.x; i <= a.nfields; i += kEncCtaThreads)
            tbase[i] = i < a.nfields ? a.fields[i].tile_base : total;
    } else {
        const huff_codebook_header *hdr = reinterpret_cast<const huff_codebook_header *>(a.one.book);
        const uint32_t nbins = hdr->nbins;
        const uint32_t max_len = hdr->max_len;
        if (max_len > kEncMaxLen || nbins != a.one.nbins) {
            if (threadIdx.x == 0) set_error(a.one.status, HUFF_ERR_INVALID_ARG);
            return;
        }
        const uint32_t nsub = enc_subs_per_tile<Sym>(max_len, a.nsub_cap);
        const uint64_t TILE = (uint64_t)enc_sub_syms<Sym>() * nsub;
        total = (uint32_t)((a.one.n + TILE - 1) / TILE);
        r = enc_clamp_r<Sym>(a.reduce_log2 >= 0 ? a.reduce_log2 : enc_rule_r(hdr->total_bits, hdr->nsymbols));
        e32 = max_len <= 23;
        nsub1 = nsub;
        max_len1 = max_len;
        if (threadIdx.x == 0) {
            S.f0 = a.one;
            S.f0.max_len = max_len;
            S.f0.nsub = nsub;
            S.f0.ntiles = total;
            S.f0.tile_base = 0;
        }
        fields = &S.f0;
    }
    for (uint32_t i = threadIdx.x; i < RW; i += kEncCtaThreads) ring[i] = 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kEncStages; s++) mbar_init(&S.bars[s], 1);
        for (int b = 0; b < kSlots; b++) {
            mbar_init(&S.full[b], 1);
            mbar_init(&S.gready[b], 1);
            mbar_init(&S.sfree[b], 1);
        }
        S.ring_tail = 0;
        fence_barrier_init();
    }
    // the kernel's first kEncCtaThreads threads (a launch may have more, idle)
    asm volatile("bar.sync 2, %0;" ::"n"(kEncCtaThreads) : "memory");
    if (threadIdx.x >= kEncThreads + 32) {
        writeout_loop<Sym>(fields, ring, total, S);
        return;
    }
    if (threadIdx.x >= kEncThreads) {
        lookback_loop(a, fields, total, S);
        return;
    }
    // a codebook outside shared memory is read from a.etab (the 32-bit entries
    // of a single field, TAB 2) or converted from its codewords (TAB 1)
    constexpr int kTab = GTAB ? 1 : 0;
    if (e32) {
        bool done = false;
        if constexpr (GTAB && !BATCH) {
            if (a.etab) {
                merge_dispatch<Sym, uint32_t, 2, BATCH, CALIGN>(r, a, fields, tbase, stage, ring, const_cast<uint32_t *>(a.etab),
                                                        total, nsub1, max_len1, S);
                done = true;
            }
        }
        if (!done)
            merge_dispatch<Sym, uint32_t, kTab, BATCH, CALIGN>(r, a, fields, tbase, stage, ring,
                                                       GTAB ? nullptr : reinterpret_cast<uint32_t *>(tab), total, nsub1,
                                                       max_len1, S);
    } else {
        merge_dispatch<Sym, uint64_t, kTab, BATCH, CALIGN>(r, a, fields, tbase, stage, ring, GTAB ? nullptr : tab, total, nsub1,
                                                   max_len1, S);
    }
}

template <typename Sym, bool GTAB, bool BATCH, bool CALIGN = false>
__global__ void __launch_bounds__(kEncCtaThreads, sizeof(Sym) == 1 ? 2 : 3) encode_kernel(EncArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ EncShared S;
    encode_body<Sym, GTAB, BATCH, CALIGN>(a, smem, S);
}

// The single-field kernel with the chunk-aligned layout's padding in the
// tile scan (instantiated in encode_aligned.cu, apart from the dense kernels).
using EncKernelFn = void (*)(EncArgs);
template <typename Sym>
EncKernelFn encode_kernel_aligned(bool gtab);

}  // namespace huff
