// Records and launch functions shared between libhuff's translation units.
// Every record here lives in device memory or is passed by value to a kernel;
// the host fills the caller-known members.
#pragma once

#include "common.cuh"

namespace huff {

// ---------------------------------------------------------------- histogram

// One field of a batched histogram, and one tile of its symbols.
struct HistField {
    const uint8_t *sym;
    uint32_t *hist;           // nbins counts, zeroed before the launch
    uint32_t *status;
    uint32_t nbins;
    uint32_t head;            // symbols before the first 16-byte aligned address (< one vector)
};

struct HistTile {
    uint32_t field;
    uint32_t pad;
    uint64_t start;           // symbols [start, end) of the field; start is a multiple of the tile size
    uint64_t end;
};

huff_status histogram_launch(const void *d_sym, uint64_t n, huff_dtype dtype, uint32_t nbins, uint32_t *d_hist,
                             uint32_t *status, cudaStream_t st);
// Symbols per tile of a batched histogram (a multiple of every vector width).
uint64_t histogram_batch_tile(uint32_t max_nbins);
huff_status histogram_batch_prepare(huff_dtype dtype, uint32_t max_nbins, int *ctas_per_sm);
huff_status histogram_batch_launch(huff_dtype dtype, const HistTile *d_tiles, uint32_t ntiles,
                                   const HistField *d_fields, uint32_t max_nbins, uint32_t grid, cudaStream_t st);

// ---------------------------------------------------------------- codebook

struct CbArgs {
    const uint32_t *hist;
    uint32_t nbins;
    uint8_t *book;         // codebook buffer
    uint8_t *scratch;      // global scratch (large alphabets)
    uint32_t *status;
};

huff_status codebook_launch(const uint32_t *d_hist, uint32_t nbins, void *d_codebook, uint8_t *scratch,
                            uint32_t *status, cudaStream_t st);
size_t codebook_scratch_bytes(uint32_t nbins);
size_t codebook_array_bytes(uint32_t nbins);
size_t codebook_batch_smem(uint32_t max_nbins);
huff_status codebook_batch_prepare(uint32_t max_nbins, int *ctas_per_sm);
huff_status codebook_batch_launch(const CbArgs *d_args, uint32_t nfields, uint32_t max_nbins, uint32_t grid,
                                  uint8_t *scratch, size_t scratch_stride, cudaStream_t st);

// ---------------------------------------------------------------- encode

// One field of an encode launch.  A single-field launch passes it by value
// and the kernel fills in the codebook-derived members; a batched launch
// keeps an array of them in device memory, completed by the batch planner.
struct EncField {
    const uint8_t *sym;
    const uint8_t *book;     // codebook buffer
    uint32_t *out;
    uint64_t *offs;
    uint64_t *total_bits;
    uint32_t *status;        // sticky first error of this field
    uint64_t n;
    uint64_t cap_words;
    uint64_t nchunks;
    uint32_t nbins;
    int32_t chunk_log2;
    uint32_t aligned;        // 16-byte aligned input: full sub-tiles use bulk copies
    // from the codebook
    uint32_t max_len;
    uint32_t nsub;           // sub-tiles per tile
    uint32_t ntiles;
    uint32_t tile_base;      // global id of the field's first tile
    uint32_t format;         // stream format (fmt_* below); 0 = dense 32-bit words
    uint32_t *etab;          // batched segment form: room for the field's 32-bit codebook entries
};

// EncField::format: bits 0-1 code the unit width W (0: 32, 1: 16, 2: 8 bits),
// bit 8 the chunk-aligned layout (every chunk starts at a unit boundary).
__host__ __device__ inline uint32_t fmt_wlog(uint32_t f) { return 5u - (f & 3u); }
__host__ __device__ inline bool fmt_chunk_aligned(uint32_t f) { return ((f >> 8) & 1u) != 0; }

// Launch-wide values of a batched encode, written by the planner on the device.
struct EncBatchConf {
    uint32_t total_tiles;
    int32_t r;               // reduction factor for every field
    uint32_t entry32;        // every codeword fits the 32-bit table entry
    uint32_t seg_total;      // batched segment form: its tiles over all the fields it takes
    int32_t seg_r;           // ... and its reduction factor (by rule over those fields)
    uint32_t seg_long;       // ... some of those fields has codewords over 23 bits
};

// Checks the format fields of p (word_bits, layout, with chunk_log2 and merge)
// for dtype and returns the EncField::format code in *fmt.
huff_status encode_format_of(const huff_params &p, huff_dtype dtype, uint32_t *fmt);
// cap counts units of the format's W bits.
huff_status encode_launch(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook, uint32_t nbins,
                          int chunk_log2, int reduce_log2, uint32_t format, uint32_t *d_out, uint64_t cap,
                          uint64_t *d_offs, uint64_t *d_total, uint8_t *scratch, uint32_t *status, cudaStream_t st);
// The same with two failure-detection knobs: id_offset is added to every tile
// id the encoder takes (1 leaves tile 0 unencoded, so the look-back of tile 1
// can only give up), and spin_limit bounds the look-back's polls (0: the
// default limit).  scratch_zeroed: the caller has cleared the scratch (the
// batched plan clears every field's with one memset).  min_tiles_per_cta: the
// grid holds at most one CTA per that many tiles (concurrent launches of
// many fields share the GPU; a CTA's start-up is paid once per CTA).
// long_ok: the kernel instance whose segment path also takes codewords over
// 23 bits (batched per-field launches; the plain instance keeps the common
// loop's registers).
huff_status encode_launch_ex(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook, uint32_t nbins,
                             int chunk_log2, int reduce_log2, uint32_t format, uint32_t *d_out, uint64_t cap,
                             uint64_t *d_offs, uint64_t *d_total, uint8_t *scratch, uint32_t *status, cudaStream_t st,
                             uint32_t id_offset, uint32_t spin_limit, bool scratch_zeroed = false,
                             uint32_t min_tiles_per_cta = 1, bool long_ok = false);
size_t encode_scratch_bytes(uint64_t n, uint32_t nbins);
// Kernel launches of one encode_launch_ex call on a non-empty field.
uint32_t encode_kernels_per_call(uint32_t nbins);
// Sets the launch attributes encode_launch_ex (long_ok) needs for a dense
// field of this dtype and alphabet size, so that later launches can be
// captured.
huff_status encode_prepare(huff_dtype dtype, uint32_t nbins);
int encode_run_log2(huff_dtype dtype);
// Symbols per sub-tile (the smallest tile) of a dtype.
uint32_t encode_sub_symbols(huff_dtype dtype);
// Reduction factors the encoder supports for a dtype.
void encode_r_range(huff_dtype dtype, int *r_min, int *r_max);
huff_status encode_batch_prepare(huff_dtype dtype, uint32_t max_nbins, uint32_t nfields, int *ctas_per_sm);
// Batched segment form (encode_seg.cuh): symbols per merge thread and per
// tile; launch attributes; the entry tables and the persistent launch over
// the segment tiles the planner laid out in seg_first.
uint32_t encode_seg_lane_symbols(huff_dtype dtype);
uint32_t encode_seg_tile_symbols(huff_dtype dtype);
huff_status encode_seg_batch_prepare(huff_dtype dtype, uint32_t nfields);
huff_status encode_seg_batch_launch(huff_dtype dtype, const EncField *d_fields, uint32_t nfields,
                                    const EncBatchConf *d_conf, const uint32_t *seg_first, uint32_t max_nbins,
                                    uint8_t *scratch, uint32_t grid, bool many, cudaStream_t st);
// seg_first (nfields + 1 entries, or null): plan the batched segment form too.
huff_status encode_batch_plan_launch(huff_dtype dtype, EncField *d_fields, uint32_t nfields, EncBatchConf *d_conf,
                                     int r_override, uint32_t nsub_cap, cudaStream_t st,
                                     uint32_t *seg_first = nullptr);
huff_status encode_batch_launch(huff_dtype dtype, const EncField *d_fields, uint32_t nfields,
                                const EncBatchConf *d_conf, uint32_t max_nbins, uint8_t *scratch, uint32_t grid,
                                cudaStream_t st);

// The paper's three-kernel encode (merge = HUFF_MERGE_SHUFFLE).
size_t shuffle_scratch_bytes(uint64_t n, int chunk_log2, int reduce_log2);
huff_status encode_shuffle_launch(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook,
                                  uint32_t nbins, int chunk_log2, int reduce_log2, uint32_t max_len, uint32_t *d_out,
                                  uint64_t cap, uint64_t *d_offs, uint64_t *d_total, uint8_t *scratch,
                                  uint32_t *status, cudaStream_t st);

// ---------------------------------------------------------------- decode

// format as EncField::format: d_in holds units of W bits; chunk-aligned
// offsets count units.
huff_status decode_launch(const void *d_in, uint64_t total_bits, const uint64_t *d_offs, int chunk_log2,
                          uint32_t format, uint64_t n, huff_dtype dtype, const void *d_codebook, uint32_t nbins,
                          void *d_out, uint32_t *status, cudaStream_t st);

}  // namespace huff
