/*
 * libhuff: GPU Huffman encoding for sm_103a (GB300).
 *
 * The operations follow the encoder of "Revisiting Huffman Coding: Toward
 * Extreme Performance on Modern GPU Architectures" (Tian et al.), whose
 * problem statement (Sec. IV, introduction) splits encoding into four stages:
 * a histogram of the input symbols, construction of a Huffman codebook from
 * it, canonisation with the reverse (decode) tables, and encoding into one
 * bitstream.  Each stage is one call below; the batched and served forms run
 * the same stages over many inputs.
 *
 * Conventions shared by every call:
 *  - Buffers named d_* are DEVICE pointers owned by the caller.  The library
 *    never frees or keeps them beyond the call (the batch plan and the server
 *    keep the pointers the caller registers with them, see there).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Compute calls are asynchronous and stream ordered; they never
 *    synchronise with the host unless stated.
 *  - Host-checkable errors (NULL pointers, unsupported sizes, dtype/nbins
 *    mismatch) return immediately with no work enqueued.
 *  - Data-dependent errors found on the device (a symbol >= nbins, a symbol
 *    without codeword, too small an output buffer, a histogram summing to
 *    2^32 or more, a device wait that gave up) are recorded as the FIRST
 *    error in a sticky status word at the start of the caller's workspace;
 *    kernels skip the offending writes and finish.  huff_get_status() reads
 *    the word (it synchronises the stream).
 *  - Symbols are little-endian unsigned integers of 1, 2 or 4 bytes; every
 *    typed device array must be aligned to its element size (a misaligned
 *    pointer returns HUFF_ERR_INVALID_ARG).
 *  - The bitstream is an array of uint32 words: bit 31 of word 0 is the first
 *    stream bit, codewords are written most significant bit first, one after
 *    another in input order (the paper's Merge operator, Sec. IV-C, places
 *    a_{2k+1} right after a_{2k}); bits after the last codeword are zero.
 */
#ifndef HUFF_H
#define HUFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { HUFF_U8 = 1, HUFF_U16 = 2, HUFF_U32 = 4 } huff_dtype;

typedef enum {
    HUFF_OK = 0,
    HUFF_ERR_INVALID_ARG = 1,      /* bad pointer, size or parameter                      */
    HUFF_ERR_SYMBOL_RANGE = 2,     /* an input symbol is >= nbins                         */
    HUFF_ERR_NOT_IN_CODEBOOK = 3,  /* an input symbol has no codeword (zero count)        */
    HUFF_ERR_CAPACITY = 4,         /* the output buffer is too small                      */
    HUFF_ERR_OOM = 5,              /* a library-owned allocation failed                   */
    HUFF_ERR_TIMEOUT = 6,          /* a bounded device wait gave up                       */
    HUFF_ERR_BUSY = 7,             /* the server has no room for the request              */
    HUFF_ERR_CUDA = 8,             /* a CUDA runtime call failed                          */
    HUFF_ERR_HIST_OVERFLOW = 9,    /* histogram counts sum to 2^32 or more                */
    HUFF_ERR_NOT_FOUND = 10,       /* unknown ticket                                      */
    HUFF_ERR_CANCELLED = 11        /* request dropped because the server shut down       */
} huff_status;

#define HUFF_MAX_LEN 64            /* codeword lengths are 1..HUFF_MAX_LEN               */
#define HUFF_MAX_BINS 1048576      /* alphabet sizes are 1..HUFF_MAX_BINS (2^20; above 65,536
                                      for HUFF_U32 symbols only)                          */
#define HUFF_MAX_BINS_BATCH 65536  /* alphabet limit of the batched, served and
                                      allocation-free forms                               */
#define HUFF_CW_LEN_SHIFT 58       /* cw = code | (len << 58)                             */

/*
 * Codebook: one caller-allocated device buffer of huff_codebook_bytes(nbins)
 * bytes, 16-byte aligned, laid out as
 *     huff_codebook_header
 *     uint64_t cw[nbins]           cw[s] = code | (len << 58); 0 = no codeword
 *     uint32_t sorted_syms[nbins]  used symbols by (length, id); nused valid
 * first/entry/count are indexed by code length (slot 0 unused):
 *     count[l]  number of codewords of length l
 *     first[l]  the numerically first (smallest) codeword of length l; every
 *               l-bit prefix of a longer codeword is below it (Sec. IV-B2)
 *     entry[l]  number of codewords shorter than l (index into sorted_syms)
 * Codewords of one length are consecutive integers in ascending symbol id.
 */
typedef struct {
    uint32_t nbins;
    uint32_t max_len;              /* 0 when no symbol is used                            */
    uint64_t first[HUFF_MAX_LEN + 1];
    uint32_t entry[HUFF_MAX_LEN + 1];
    uint32_t count[HUFF_MAX_LEN + 1];
    uint32_t nused;
    uint32_t status;               /* huff_status of the build (HUFF_OK or an error)     */
    uint64_t total_bits;           /* sum over symbols of count * length: encoded size   */
    uint64_t nsymbols;             /* sum of the counts the codebook was built from      */
} huff_codebook_header;

/* Encoder tunables (Sec. IV-C "Interface": ReduceShuffleMerge<M, r>). */
typedef struct {
    int32_t chunk_log2;    /* M: one chunk offset per 2^M symbols; 4..30; paper default 10     */
    int32_t reduce_log2;   /* r: 2^r consecutive symbols merged per thread in registers;
                              -1 = pick r from the average codeword length (Sec. IV-C rule,
                              as huff_reduce_factor with 32-bit words).  Whatever r is asked
                              for or ruled, the scan encoder then clamps it to what its
                              registers allow: [2, 4] for u8, [2, 3] for u16, and for u32
                              [1, 2] on its segment path (codes of at most 23 bits), [0, 2]
                              otherwise; the shuffle encoder takes r as given (<= 4; -1 = 3,
                              fixed).  r never changes the output                             */
    int32_t block_threads; /* reserved: the encoders' CTA shapes are fixed per dtype (the
                              autotuner of the batched form picks CTAs per SM); any value is
                              accepted and ignored                                            */
    int32_t merge;         /* HUFF_MERGE_*                                                    */
    int32_t word_bits;     /* W, the typed unit of the stream (Sec. IV-C: uint{8,16,32} data
                              cells): 8, 16 or 32 (0 = 32).  The stream is an array of W-bit
                              units, bit W-1 of unit 0 first; W also replaces 32 in the r
                              rule (huff_reduce_factor(beta, W)).  8 and 16 need the scan
                              encoder (merge AUTO or SCAN)                                    */
    int32_t layout;        /* HUFF_LAYOUT_*                                                   */
} huff_params;

enum {
    HUFF_LAYOUT_DENSE = 0,          /* one bit-contiguous stream; offsets count bits           */
    HUFF_LAYOUT_CHUNK_ALIGNED = 1   /* the chunks before the optional dense gathering (Sec. VI):
                                       every chunk of 2^M symbols starts at a W-bit unit, its
                                       last unit zero-padded; offsets count units.  Needs the
                                       scan encoder and M within one encoder sub-tile and at
                                       least one warp's symbols: 10..13 for u8, 9..12 for u16,
                                       8..11 for u32                                          */
};

enum {
    HUFF_MERGE_AUTO = 0,     /* = HUFF_MERGE_SCAN                                                */
    HUFF_MERGE_SCAN = 1,     /* one fused kernel: scan of merged lengths, one placement in shared
                                memory, decoupled look-back and write-out of the dense stream      */
    HUFF_MERGE_SHUFFLE = 2   /* the paper's layout: per chunk of 2^M symbols, reduce-merge and
                                M - r log steps of shuffle-merge in shared memory into a chunk
                                slot of the workspace, then a scan of chunk lengths and a
                                coalescing copy (three kernels).  Needs r <= 4 (-1 = 3) and
                                M - r <= 10, and a workspace sized with these parameters      */
};

/* Fills *p with the defaults (M = 10, r = auto, block = 0, merge = auto, W = 32,
   dense layout). */
void huff_default_params(huff_params *p);

/*
 * Reduction factor rule of Sec. IV-C: floor(log2 beta) + r + 1 = log2(word_bits),
 * solved for r and clamped to [0, log2(word_bits)]; beta = average codeword
 * length in bits (> 0, else 3 is returned).  This is the rule's value; the
 * encoders' own clamps (see huff_params.reduce_log2) apply after it.
 */
int huff_reduce_factor(double avg_bits, int word_bits);

/* Bytes of the codebook buffer for an alphabet of nbins symbols. */
size_t huff_codebook_bytes(uint32_t nbins);

/* Bytes of output (uint32 words) that always suffice: ceil(n * max_len / 32). */
uint64_t huff_max_output_words(uint64_t n, uint32_t max_len);

/* Units of W = p->word_bits bits that always suffice for the stream of n
 * symbols in p's format: ceil(n * max_len / W), plus one unit per chunk for
 * the padding of the chunk-aligned layout (p = NULL: defaults). */
uint64_t huff_max_output_units(uint64_t n, uint32_t max_len, const huff_params *p);

/*
 * Bytes of device workspace one histogram/codebook/encode sequence needs for
 * inputs of up to n symbols over nbins bins with parameters *p (NULL =
 * defaults).  The first 256 bytes hold the sticky status word.
 */
size_t huff_workspace_bytes(uint64_t n, uint32_t nbins, const huff_params *p);

/* Clears the status word of a workspace (stream ordered).  Call once after allocating it. */
huff_status huff_workspace_init(void *d_ws, void *stream);

/*
 * Histogram (Sec. IV-A): d_hist[k] = number of i < n with d_sym[i] == k.
 *   d_sym   n symbols of `dtype`, aligned to the element size (16-byte aligned is fastest)
 *   n       < 2^32; 0 gives an all-zero histogram
 *   nbins   1..HUFF_MAX_BINS (<= 256 for HUFF_U8, <= 65536 for HUFF_U16)
 *   d_hist  nbins uint32, overwritten
 * A symbol >= nbins records HUFF_ERR_SYMBOL_RANGE and is not counted.
 */
huff_status huff_histogram(const void *d_sym, uint64_t n, huff_dtype dtype, uint32_t nbins,
                           uint32_t *d_hist, void *d_ws, void *stream);

/*
 * Codebook (Sec. IV-B, Algorithm 1): optimal Huffman code lengths for every
 * symbol with a nonzero count, then canonical codewords and the First/Entry
 * decode metadata, written to d_codebook (layout above).
 * Ties: leaves ordered by (count, id); when a leaf and a joined node weigh
 * the same the leaf is joined first (the two-queue rule); the result equals
 * the serial two-queue construction bit for bit.
 *   d_hist      nbins uint32 counts whose sum must be < 2^32
 *   d_codebook  huff_codebook_bytes(nbins) bytes, 16-byte aligned
 * A sum >= 2^32 records HUFF_ERR_HIST_OVERFLOW and writes an empty codebook.
 */
huff_status huff_build_codebook(const uint32_t *d_hist, uint32_t nbins, void *d_codebook,
                                void *d_ws, void *stream);

/*
 * Encode (Sec. IV-C, reduce-merge and shuffle-merge; gathering into one dense
 * stream as in Table I's "get blockwise code len" and "coalescing copy"):
 *   d_sym              n symbols (< 2^32) of `dtype`
 *   d_codebook         a codebook built for the same alphabet
 *   nbins              its alphabet size (checked against the codebook on the device)
 *   p                  tunables (NULL = defaults); chunk_log2, word_bits and layout
 *                      choose the format, the others never change the output
 *   d_out              4-byte aligned; out_capacity_words units of W bits (uint32
 *                      words for the default W = 32); receives ceil(total_bits/W)
 *                      units.  With W < 32 the allocation must extend to a whole
 *                      number of 32-bit words (the decoder reads whole words)
 *   d_chunk_bit_offset ceil(n / 2^M) + 1 uint64: dense layout, bit position of
 *                      symbol c*2^M and last entry total_bits; chunk-aligned
 *                      layout, unit index of chunk c and last entry the units
 *   d_total_bits       one uint64: the stream's bits (chunk-aligned: with padding)
 * A symbol >= nbins or without codeword records an error; so does a stream
 * longer than the capacity (nothing is written past it).
 */
huff_status huff_encode(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook,
                        uint32_t nbins, const huff_params *p, uint32_t *d_out, uint64_t out_capacity_words,
                        uint64_t *d_chunk_bit_offset, uint64_t *d_total_bits,
                        void *d_ws, void *stream);

/*
 * Decode (Sec. IV-B2, treeless canonical decoding with First and Entry): one
 * thread per chunk walks the stream from d_chunk_bit_offset[c] to
 * d_chunk_bit_offset[c + 1] (the layout huff_encode writes).
 *   d_in        stream words (uint32, MSB first), ceil(total_bits / 32) of them;
 *               4-byte aligned
 *   chunk_log2  M of the encode (2^M symbols per chunk), 0..30
 *   d_codebook  the codebook the stream was encoded with (nbins must match)
 *   d_out       n symbols of `dtype`, aligned to the element size; 8- or
 *               16-byte alignment (with 2^M * sizeof(sym) a multiple of it)
 *               enables wider stores
 * Host-side argument errors return immediately.  On the device, a window
 * that starts no codeword, or a chunk whose codes do not end exactly at the
 * next chunk's offset, records HUFF_ERR_INVALID_ARG in the workspace status
 * (huff_get_status); reads stay inside the stream and writes inside the
 * chunk's n symbols whatever the stream holds, and a chunk stops at its
 * first invalid code.  A corrupted stream that still parses into valid codes
 * may decode to other symbols without an error.
 */
huff_status huff_decode(const uint32_t *d_in, uint64_t total_bits, const uint64_t *d_chunk_bit_offset,
                        int chunk_log2, uint64_t n, huff_dtype dtype, const void *d_codebook,
                        uint32_t nbins, void *d_out, void *d_ws, void *stream);

/*
 * huff_decode for any format huff_encode writes: p's chunk_log2, word_bits
 * and layout must be those of the encode (p = NULL: defaults, the same as
 * huff_decode).  d_in holds the units (4-byte aligned, readable to a whole
 * number of 32-bit words); d_chunk_bit_offset and total_bits are the
 * encode's, in its units.  In the chunk-aligned layout a chunk's codes must
 * end within the last unit before the next chunk's offset.
 */
huff_status huff_decode_ex(const void *d_in, uint64_t total_bits, const uint64_t *d_chunk_bit_offset,
                           const huff_params *p, uint64_t n, huff_dtype dtype, const void *d_codebook,
                           uint32_t nbins, void *d_out, void *d_ws, void *stream);

/*
 * Encode without any device allocation by the library or the caller's
 * workspace.  The paper has no counterpart: this exists for callers that
 * cannot allocate device memory -- e.g. code running inside another
 * framework that owns every device allocation, or a loop that must not call
 * cudaMalloc/cudaFree because they can synchronise the whole device.
 * Same arguments and output as huff_encode, except:
 *   - no d_ws: the encoder's scratch is a fixed device array inside the
 *     library (2 MiB + 256 KiB + 256 bytes, held on every GPU that loads the
 *     library until the process exits);
 *   - n may be at most 2^28 symbols (268,435,456); more returns
 *     HUFF_ERR_INVALID_ARG with nothing enqueued;
 *   - p->merge must be HUFF_MERGE_AUTO or HUFF_MERGE_SCAN (the paper-layout
 *     merge needs chunk slots the fixed array does not hold): any other
 *     value returns HUFF_ERR_INVALID_ARG;
 *   - d_status: one caller-owned uint32 in device memory; the call sets it to
 *     0 and the kernel records the first device error there (huff_status
 *     codes), which the caller reads after synchronising.
 * The array's device address is looked up on every call made outside a
 * stream capture (so calls after a cudaDeviceReset use the new context's
 * array); a call inside a capture reuses the address of the last uncaptured
 * call on the same device, so the first call on a device must come before
 * any capture (else HUFF_ERR_INVALID_ARG).  Every call uses the same array
 * and clears what it needs first, so calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 */
huff_status huff_encode_noalloc(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook,
                                uint32_t nbins, const huff_params *p, uint32_t *d_out, uint64_t out_capacity_words,
                                uint64_t *d_chunk_bit_offset, uint64_t *d_total_bits, uint32_t *d_status,
                                void *stream);

/* Failure-detection test hook (no paper counterpart): huff_encode with the
 * default parameters, except that the encoder's tile ids start at 1, so tile 0
 * is never encoded and never publishes its descriptor, and the decoupled
 * look-back (Sec. IV-B's prefix sum done in one pass) gives up after
 * `poll_limit` polls (1..2^22) instead of the default 2^22.  The look-back of
 * tile 1 therefore must give up: the launch still completes, the workspace
 * status reads HUFF_ERR_TIMEOUT, and the output stream is invalid (writes stay
 * within out_capacity_words).  Requires n above eight encode sub-tiles (the
 * largest tile), so that there is a tile 1; else HUFF_ERR_INVALID_ARG.  Arguments as in
 * huff_encode.  For tests of the bounded waits only. */
huff_status huff_encode_fault_test(const void *d_sym, uint64_t n, huff_dtype dtype, const void *d_codebook,
                                   uint32_t nbins, uint32_t *d_out, uint64_t out_capacity_words,
                                   uint64_t *d_chunk_bit_offset, uint64_t *d_total_bits, uint32_t poll_limit,
                                   void *d_ws, void *stream);

/* ------------------------------------------------------------------------
 * Batched encoding.  The paper encodes one field per call; the batch form
 * (no paper counterpart) runs the histogram, codebook and encode stages of
 * many independent fields as a handful of launches captured once in a CUDA
 * graph: one histogram launch over all fields' tiles, one codebook launch
 * with a CTA per field, a one-CTA planner that lays out every field's encode
 * tiles from its codebook, and ONE persistent encode launch whose tiles run
 * over all fields (each field keeps its own stream, offsets and look-back).
 * Fields are grouped by dtype and alphabet class (<= 4,096 / <= 16,384 /
 * larger), at most 512 per group; each group adds one such launch set.
 * ------------------------------------------------------------------------ */
typedef struct {
    const void *d_sym;              /* n symbols of dtype, element aligned                            */
    uint64_t n;                     /* < 2^32                                                         */
    huff_dtype dtype;
    uint32_t nbins;                 /* 1..HUFF_MAX_BINS_BATCH (<= 256 for HUFF_U8)                    */
    int32_t chunk_log2;             /* M, 4..30; -1 = chosen by the plan from {10, 12, 14}: size the
                                       offsets for M = 10                                            */
    uint32_t reserved;
    uint32_t *d_out;                /* out_capacity_words uint32                                      */
    uint64_t out_capacity_words;
    uint64_t *d_chunk_bit_offset;   /* ceil(n / 2^M) + 1 uint64                                       */
    uint64_t *d_total_bits;         /* one uint64                                                     */
} huff_field;

typedef struct {
    int32_t autotune;       /* 1: time candidate settings on the fields at plan creation, keep the fastest */
    int32_t reduce_log2;    /* r for every field, -1 = the Sec. IV-C rule on the group's mean codeword
                               length (used when not tuning)                                            */
    int32_t max_subtiles;   /* sub-tiles per encode tile, 1..8; 0 = 8 (used when not tuning)             */
    int32_t ctas_per_sm;    /* encode CTAs per SM; 0 = as many as fit (used when not tuning)            */
    int32_t encode_form;    /* 0: the encode stage is one persistent launch of the general encoder over
                               all fields of a group;
                               1: one single-field encode launch per field (as huff_encode: the segment
                               encoder where a field's codewords allow it), run concurrently on the
                               plan's side streams inside the graph;
                               2: one persistent launch of the segment encoder over the fields whose
                               codewords fit it (at most 23 bits), then the general encoder over the
                               rest (used when not tuning; the tuner times all three)                */
} huff_batch_cfg;

typedef struct {
    int32_t reduce_log2;     /* setting in use (-1 = rule)                                        */
    int32_t max_subtiles;
    int32_t ctas_per_sm;
    int32_t chunk_log2;      /* M given to fields created with -1 (0: no such field)               */
    uint32_t groups;         /* launch groups                                                     */
    uint32_t kernels_per_run;/* kernel launches per huff_batch_encode                             */
    uint32_t candidates;     /* settings timed by the tuner (0: not tuned)                        */
    float tuned_ms;          /* best time of one batch during tuning                              */
    uint64_t device_bytes;   /* device memory held by the plan                                    */
    uint32_t encode_form;    /* encode form in use (huff_batch_cfg.encode_form)                   */
    uint32_t per_field_tiles;/* per-field form: least tiles per CTA of each launch (0: not in use)  */
} huff_batch_info;

typedef struct huff_batch_plan huff_batch_plan;

/* Default configuration: autotune off, r by rule, 8 sub-tiles, CTAs that fit, one persistent encode launch. */
void huff_batch_default_cfg(huff_batch_cfg *cfg);

/*
 * Builds a plan for nfields fields (1..65536).  The plan copies the records;
 * their device buffers must stay valid while the plan is used, and their
 * contents may change between runs.  It allocates its own device memory
 * (histograms, codebooks, tile tables, look-back descriptors) and captures
 * the launches in a CUDA graph.  With cfg->autotune it runs the batch for
 * every candidate setting (outputs are the same for all of them) and keeps
 * the fastest.  Work is done on `stream`, which is synchronised on return.
 */
huff_status huff_batch_plan_create(const huff_field *fields, uint32_t nfields, const huff_batch_cfg *cfg,
                                   void *stream, huff_batch_plan **out);

/* Runs the whole batch: one graph launch on `stream` (asynchronous). */
huff_status huff_batch_encode(huff_batch_plan *plan, void *stream);

/*
 * Measurement aid: runs the plan's launch sequence once on `stream` WITHOUT
 * the graph, with events between stages, synchronises, and writes the device
 * time in ms of each stage summed over groups: stage_ms[0] histogram,
 * [1] codebooks, [2] tile planner (+ scratch clear), [3] encode.  The outputs
 * are the same as huff_batch_encode's.
 */
huff_status huff_batch_profile(huff_batch_plan *plan, void *stream, float *stage_ms);

/* Synchronises `stream` and copies each field's first device error (huff_status) into h_status[nfields]. */
huff_status huff_batch_status(huff_batch_plan *plan, uint32_t *h_status, void *stream);

huff_status huff_batch_get_info(const huff_batch_plan *plan, huff_batch_info *info);

/* Device pointers of a field's codebook and histogram, owned by the plan (valid until destroy). */
const void *huff_batch_codebook(const huff_batch_plan *plan, uint32_t field);
const uint32_t *huff_batch_histogram(const huff_batch_plan *plan, uint32_t field);

/* The M a field is encoded with (-1 for a bad field index). */
int huff_batch_chunk_log2(const huff_batch_plan *plan, uint32_t field);

/* Frees the plan after synchronising the device work it may still have in flight. */
void huff_batch_plan_destroy(huff_batch_plan *plan);

/* ------------------------------------------------------------------------
 * Served form (no paper counterpart): a request loop on one GPU.  Clients
 * submit encode jobs whose symbols are already in device memory; a
 * dispatcher thread admits them in arrival order while the server's device
 * memory budget and in-flight limit allow, and launches every group of
 * admitted jobs as one batch (the batched histogram, codebook, planner and
 * encode kernels) on the next free stream context, so jobs that arrive while
 * others run are batched and overlap with them on the device (continuous
 * batching).  Each job's codebook, stream and chunk offsets are written to
 * server memory that stays valid until the client releases the ticket.
 * Results are identical to the plain calls on the same input.
 * ------------------------------------------------------------------------ */
typedef struct {
    uint64_t mem_budget_bytes;   /* device memory for job results (codebook, stream, offsets)          */
    uint32_t max_inflight;       /* jobs admitted and not yet released (0 = 4096)                      */
    uint32_t nstreams;           /* batches that may run at once, one stream each (0 = 2)               */
    uint32_t max_batch;          /* jobs per batch (1..512, 0 = 64)                                     */
    int32_t chunk_log2;          /* M of every job (0 = 10)                                             */
    uint64_t max_batch_symbols;  /* symbols per batch (0 = 2^31)                                        */
    uint32_t max_queue;          /* jobs waiting for admission before submit returns BUSY (0 = 1<<20)   */
    uint32_t reserved;
} huff_serve_cfg;

typedef struct {
    const void *d_sym;           /* n symbols of dtype in device memory, element aligned; must stay
                                    unchanged until the job is done                                  */
    uint64_t n;                  /* 1 .. max_batch_symbols                                            */
    huff_dtype dtype;
    uint32_t nbins;
} huff_request;

typedef struct {
    huff_status status;          /* HUFF_OK or the job's first device error (or CANCELLED)            */
    int32_t chunk_log2;
    uint64_t total_bits;
    const uint32_t *d_out;       /* ceil(total_bits / 32) words (server memory)                       */
    const uint64_t *d_chunk_bit_offset;   /* ceil(n / 2^M) + 1 offsets (server memory)               */
    const void *d_codebook;      /* the job's codebook (layout above, server memory)                  */
    double t_submit, t_admit, t_launch, t_done;   /* seconds on the server's steady clock             */
} huff_result;

typedef struct {
    uint64_t submitted, completed, cancelled, batches;
    uint64_t max_batch_jobs;     /* largest batch launched                                            */
    uint32_t max_concurrent_batches;   /* most batches on the device at once                        */
    uint32_t reserved;
    uint64_t pool_used, pool_peak, pool_capacity;
    uint64_t symbols_done;
} huff_serve_stats;

typedef struct huff_server huff_server;

void huff_serve_default_cfg(huff_serve_cfg *cfg);

/* Creates the server on the current device: allocates the budget and the stream contexts. */
huff_status huff_serve_create(const huff_serve_cfg *cfg, huff_server **out);

/*
 * Queues a job; *ticket identifies it.  HUFF_ERR_INVALID_ARG for a bad
 * request, HUFF_ERR_OOM if its results could never fit the budget,
 * HUFF_ERR_BUSY if the admission queue is full (nothing queued).
 */
huff_status huff_serve_submit(huff_server *srv, const huff_request *req, uint64_t *ticket);

/* HUFF_OK and *res if the job is done (or cancelled); HUFF_ERR_BUSY while it is
   pending; HUFF_ERR_NOT_FOUND for an unknown or released ticket. */
huff_status huff_serve_poll(huff_server *srv, uint64_t ticket, huff_result *res);

/* Blocks until the job is done (or cancelled), then as huff_serve_poll. */
huff_status huff_serve_wait(huff_server *srv, uint64_t ticket, huff_result *res);

/* Frees the job's result memory; its result pointers become invalid.  A job
   still pending is released as soon as it completes. */
huff_status huff_serve_release(huff_server *srv, uint64_t ticket);

huff_status huff_serve_get_stats(huff_server *srv, huff_serve_stats *stats);

/* Cancels jobs not yet launched, waits for the launched ones, frees everything. */
huff_status huff_serve_destroy(huff_server *srv);

/* Synchronises `stream` and returns the first device error recorded in d_ws. */
huff_status huff_get_status(const void *d_ws, void *stream);

/* Short text for a status code (static storage). */
const char *huff_status_string(huff_status s);

/* Number of kernel launches this library has issued in this process. */
uint64_t huff_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* HUFF_H */
