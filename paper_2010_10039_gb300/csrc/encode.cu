// Single-field encode launch (huff_encode, huff_encode_noalloc): the kernel
// of encode_impl.cuh over one field whose codebook-derived tile layout the
// kernel works out itself.
#include "encode_seg.cuh"

namespace huff {

// counter + one 16-byte descriptor per tile (at most one tile per u32 sub-tile)
static size_t desc_area_bytes(uint64_t n) {
    uint64_t ntiles = (n + enc_sub_syms<uint32_t>() - 1) / enc_sub_syms<uint32_t>();
    return (64 + 16 * ntiles + 255) & ~size_t(255);
}

// ... then, for a codebook too large for shared memory, its 32-bit entries
size_t encode_scratch_bytes(uint64_t n, uint32_t nbins) {
    return desc_area_bytes(n) + (nbins > kEncSmemTableBins ? 4ull * nbins : 0);
}

// The codebook's 32-bit table entries (code << (32 - l) | l, a flag entry for
// codewords over 23 bits), precomputed once per launch when the codebook stays
// in global memory: a lookup then reads one word instead of converting a
// 64-bit codeword, and the segment path, which takes 32-bit entries, can run.
// The general encoder reads them only when every codeword has at most 23
// bits.  Up to 65,536 entries (the allocation-free entry point's array holds
// that many).
constexpr uint32_t kEncEntryTableBins = 65536;
__global__ void entry_table_kernel(const uint8_t *book, uint32_t nbins, uint32_t *etab) {
    const uint64_t *gcw = reinterpret_cast<const uint64_t *>(book + cb_cw_offset());
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nbins; i += gridDim.x * blockDim.x)
        etab[i] = seg_entry_from_cw(gcw[i]);
}

uint32_t encode_kernels_per_call(uint32_t nbins) {
    return 1u + (nbins > kEncSmemTableBins && nbins <= kEncEntryTableBins ? 1u : 0u);
}

template <typename Sym>
static huff_status prepare_one(uint32_t nbins) {
    const bool gtab = nbins > kEncSmemTableBins;
    const void *k = (!gtab || nbins <= kEncEntryTableBins) ? (const void *)encode_one_kernel_get<Sym>(gtab, true)
                                                            : (const void *)encode_kernel<Sym, true, false>;
    return allow_dynamic_smem(k, 0) ? HUFF_OK : HUFF_ERR_CUDA;
}

huff_status encode_prepare(huff_dtype dtype, uint32_t nbins) {
    switch (dtype) {
        case HUFF_U8: return prepare_one<uint8_t>(nbins);
        case HUFF_U16: return prepare_one<uint16_t>(nbins);
        case HUFF_U32: return prepare_one<uint32_t>(nbins);
    }
    return HUFF_ERR_INVALID_ARG;
}

static uint32_t pow2_at_least(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <typename Sym>
static huff_status launch_encode(const void *d_sym, uint64_t n, const void *d_codebook, uint32_t nbins_host,
                                 int chunk_log2, int reduce_log2, uint32_t format, uint32_t *d_out, uint64_t cap,
                                 uint64_t *d_offs, uint64_t *d_total, uint8_t *scratch, uint32_t *status,
                                 cudaStream_t st, uint32_t id_offset, uint32_t spin_limit, bool zeroed,
                                 uint32_t tiles_per_cta, bool long_ok) {
    constexpr uint32_t SUB = enc_sub_syms<Sym>();
    EncArgs a{};
    a.one.sym = static_cast<const uint8_t *>(d_sym);
    a.one.book = static_cast<const uint8_t *>(d_codebook);
    a.one.out = d_out;
    a.one.offs = d_offs;
    a.one.total_bits = d_total;
    a.one.status = status;
    a.one.n = n;
    a.one.cap_words = cap;
    a.one.nchunks = (n + (1ull << chunk_log2) - 1) >> chunk_log2;
    a.one.nbins = nbins_host;
    a.one.chunk_log2 = chunk_log2;
    a.one.aligned = ((uintptr_t)d_sym & 15) == 0;
    a.one.format = format;
    a.fields = nullptr;
    a.conf = nullptr;
    a.nfields = 1;
    a.tslots = pow2_at_least(nbins_host);
    a.tile_counter = reinterpret_cast<uint32_t *>(scratch);
    a.desc = reinterpret_cast<uint64_t *>(scratch + 64);
    a.reduce_log2 = reduce_log2;
    a.nsub_cap = kEncMaxSubs;
    a.id_offset = id_offset;
    a.spin_limit = spin_limit;
    const uint64_t max_tiles = (n + SUB - 1) / SUB;
    if (!zeroed && cudaMemsetAsync(scratch, 0, 64 + 16 * max_tiles, st) != cudaSuccess) return HUFF_ERR_CUDA;
    const bool gtab = nbins_host > kEncSmemTableBins;
    if (gtab && nbins_host <= kEncEntryTableBins) {
        uint32_t *etab = reinterpret_cast<uint32_t *>(scratch + desc_area_bytes(n));
        entry_table_kernel<<<(nbins_host + 255) / 256, 256, 0, st>>>(a.one.book, nbins_host, etab);
        note_launch();
        a.etab = etab;
    }
    size_t smem = enc_smem_bytes<Sym>(gtab, a.tslots, 0);
    void (*kern)(EncArgs);
    int threads = kEncCtaThreads;
    // tiles the grid is sized for: sub-tiles, or segment tiles where the
    // segment path may run (the general encoder's tiles then hold up to 8
    // sub-tiles, about a segment tile's symbols)
    uint64_t tiles = max_tiles;
    if (fmt_chunk_aligned(format)) {
        kern = encode_kernel_aligned<Sym>(gtab);
    } else if (!gtab || a.etab) {
        // the segment path when the codebook allows it (decided on the device),
        // else the general encoder: room for either layout
        kern = encode_one_kernel_get<Sym>(gtab, long_ok);
        threads = kSegThreads;
        tiles = (n + seg_sub_syms<Sym>() - 1) / seg_sub_syms<Sym>();
        const size_t seg = seg_smem_bytes<Sym>(a.tslots, gtab);
        if (seg > smem) smem = seg;
    } else {
        kern = encode_kernel<Sym, true, false>;
    }
    if (!allow_dynamic_smem((const void *)kern, smem))
        return HUFF_ERR_CUDA;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (occ < 1) occ = 1;
    uint64_t grid = (uint64_t)sm_count() * occ;
    const uint64_t per = tiles_per_cta > 1 ? tiles_per_cta : 1;
    if (grid > (tiles + per - 1) / per) grid = (tiles + per - 1) / per;
    kern<<<(unsigned)grid, threads, smem, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

huff_status encode_launch_ex(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook, uint32_t nbins,
                             int chunk_log2, int reduce_log2, uint32_t format, uint32_t *d_out, uint64_t cap,
                             uint64_t *d_offs, uint64_t *d_total, uint8_t *scratch, uint32_t *status, cudaStream_t st,
                             uint32_t id_offset, uint32_t spin_limit, bool zeroed, uint32_t tiles_per_cta,
                             bool long_ok) {
    switch (dtype) {
        case HUFF_U8: return launch_encode<uint8_t>(d_sym, n, d_codebook, nbins, chunk_log2, reduce_log2, format, d_out, cap, d_offs, d_total, scratch, status, st, id_offset, spin_limit, zeroed, tiles_per_cta, long_ok);
        case HUFF_U16: return launch_encode<uint16_t>(d_sym, n, d_codebook, nbins, chunk_log2, reduce_log2, format, d_out, cap, d_offs, d_total, scratch, status, st, id_offset, spin_limit, zeroed, tiles_per_cta, long_ok);
        case HUFF_U32: return launch_encode<uint32_t>(d_sym, n, d_codebook, nbins, chunk_log2, reduce_log2, format, d_out, cap, d_offs, d_total, scratch, status, st, id_offset, spin_limit, zeroed, tiles_per_cta, long_ok);
    }
    return HUFF_ERR_INVALID_ARG;
}

huff_status encode_launch(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook, uint32_t nbins,
                          int chunk_log2, int reduce_log2, uint32_t format, uint32_t *d_out, uint64_t cap,
                          uint64_t *d_offs, uint64_t *d_total, uint8_t *scratch, uint32_t *status, cudaStream_t st) {
    return encode_launch_ex(d_sym, n, dtype, d_codebook, nbins, chunk_log2, reduce_log2, format, d_out, cap, d_offs,
                            d_total, scratch, status, st, 0u, 0u, false, 1u, false);
}

huff_status encode_format_of(const huff_params &p, huff_dtype dtype, uint32_t *fmt) {
    const int W = p.word_bits == 0 ? 32 : p.word_bits;
    if (W != 8 && W != 16 && W != 32) return HUFF_ERR_INVALID_ARG;
    if (p.layout != HUFF_LAYOUT_DENSE && p.layout != HUFF_LAYOUT_CHUNK_ALIGNED) return HUFF_ERR_INVALID_ARG;
    const bool aligned = p.layout == HUFF_LAYOUT_CHUNK_ALIGNED;
    if ((W != 32 || aligned) && p.merge == HUFF_MERGE_SHUFFLE) return HUFF_ERR_INVALID_ARG;
    if (aligned) {
        // chunk boundaries must fall on warp boundaries of a sub-tile: the
        // padding is added to the warp totals of the tile scan
        int sub_log2 = 0;
        while ((1u << (sub_log2 + 1)) <= encode_sub_symbols(dtype)) sub_log2++;
        const int warp_log2 = sub_log2 - 3;                     // 8 merge warps per sub-tile
        if (p.chunk_log2 < warp_log2 || p.chunk_log2 > sub_log2) return HUFF_ERR_INVALID_ARG;
    }
    *fmt = (W == 32 ? 0u : W == 16 ? 1u : 2u) | (aligned ? 0x100u : 0u);
    return HUFF_OK;
}

uint32_t encode_sub_symbols(huff_dtype dtype) {
    return dtype == HUFF_U8 ? enc_sub_syms<uint8_t>() : dtype == HUFF_U16 ? enc_sub_syms<uint16_t>()
                                                                          : enc_sub_syms<uint32_t>();
}

void encode_r_range(huff_dtype dtype, int *r_min, int *r_max) {
    switch (dtype) {
        case HUFF_U8: *r_min = enc_r_min<uint8_t>(); *r_max = enc_r_max<uint8_t>(); return;
        case HUFF_U16: *r_min = enc_r_min<uint16_t>(); *r_max = enc_r_max<uint16_t>(); return;
        default: *r_min = enc_r_min<uint32_t>(); *r_max = enc_r_max<uint32_t>(); return;
    }
}

int encode_run_log2(huff_dtype dtype) {
    return dtype == HUFF_U8 ? 4 : dtype == HUFF_U16 ? 3 : 2;
}

}  // namespace huff
