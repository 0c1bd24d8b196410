// Batched encode: the planner that lays out every field's tiles once its
// codebook exists (on the device, so the whole batch runs without a host
// round trip and can be captured in a CUDA graph), and the launch of the
// encode kernel of encode_impl.cuh over all fields at once.
#include <algorithm>

#include "encode_seg.cuh"

namespace huff {

constexpr int kPlanThreads = 1024;

// Exclusive scan of one value per thread over the CTA (kPlanThreads), plus
// the running carry of earlier calls; returns this thread's prefix.
__device__ __forceinline__ uint32_t plan_scan(uint32_t v, uint32_t *s_warp, uint32_t &s_carry) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = s_warp[lane];
        uint32_t w = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w - x;
    }
    __syncthreads();
    const uint32_t excl = s_carry + s_warp[warp] + inc - v;
    __syncthreads();
    if (tid == kPlanThreads - 1) s_carry = excl + v;
    __syncthreads();
    return excl;
}

// One CTA: per field, the sub-tiles per tile from its longest codeword, the
// number of tiles and (exclusive scan) its first global tile id; then the
// launch-wide tile total, reduction factor and table entry form.  A field
// whose codebook failed, or does not fit the encoder, gets no tiles; an
// empty field gets total_bits = 0 and one offset 0 here.  With seg_first
// (the batched segment form), a field whose codewords fit the segment path
// gets segment tiles instead (first ids in seg_first, the total after the
// last field) and no tiles of the general encoder.
template <typename Sym>
__global__ void __launch_bounds__(kPlanThreads) batch_plan_kernel(EncField *fields, uint32_t nfields,
                                                                   EncBatchConf *conf, int r_override,
                                                                   uint32_t nsub_cap, uint32_t *seg_first) {
    constexpr uint32_t SUB = enc_sub_syms<Sym>();
    constexpr uint32_t SEG_SUB = seg_sub_syms<Sym>();
    __shared__ unsigned long long s_tb, s_ns, s_stb, s_sns;
    __shared__ uint32_t s_wide, s_carry, s_scarry, s_slong;
    __shared__ uint32_t s_warp[kPlanThreads / 32];
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) { s_tb = 0; s_ns = 0; s_stb = 0; s_sns = 0; s_wide = 0; s_carry = 0; s_scarry = 0; s_slong = 0; }
    __syncthreads();
    uint64_t tb = 0, ns = 0, stb = 0, sns = 0;
    uint32_t wide = 0;
    for (uint32_t c0 = 0; c0 < nfields; c0 += kPlanThreads) {
        const uint32_t i = c0 + tid;
        uint32_t nt = 0, snt = 0;
        if (i < nfields) {
            EncField &F = fields[i];
            const huff_codebook_header *hdr = reinterpret_cast<const huff_codebook_header *>(F.book);
            const uint32_t ml = hdr->max_len;
            bool ok = hdr->status == HUFF_OK;
            if (hdr->nbins != F.nbins || ml > kEncMaxLen) {
                set_error(F.status, HUFF_ERR_INVALID_ARG);
                ok = false;
            }
            F.max_len = ml;
            F.nsub = enc_subs_per_tile<Sym>(ml, nsub_cap);
            if (F.n == 0) {
                F.offs[0] = 0;
                *F.total_bits = 0;
            } else if (ok && seg_first && seg_fits<Sym>(ml) && !fmt_chunk_aligned(F.format)) {
                snt = (uint32_t)((F.n + SEG_SUB - 1) / SEG_SUB);
                if (ml > kSegEntryLen) s_slong = 1;
                stb += hdr->total_bits;
                sns += hdr->nsymbols;
            } else if (ok) {
                const uint64_t TILE = (uint64_t)SUB * F.nsub;
                nt = (uint32_t)((F.n + TILE - 1) / TILE);
                tb += hdr->total_bits;
                ns += hdr->nsymbols;
                if (ml > 23) wide = 1;
            }
            F.ntiles = nt;
        }
        if (seg_first) {
            const uint32_t sx = plan_scan(snt, s_warp, s_scarry);
            if (i < nfields) seg_first[i] = sx;
        }
        // block exclusive scan of the tile counts
        const uint32_t excl = plan_scan(nt, s_warp, s_carry);
        if (i < nfields) fields[i].tile_base = excl;
    }
    for (int o = 16; o; o >>= 1) {
        tb += __shfl_xor_sync(0xFFFFFFFFu, tb, o);
        ns += __shfl_xor_sync(0xFFFFFFFFu, ns, o);
        stb += __shfl_xor_sync(0xFFFFFFFFu, stb, o);
        sns += __shfl_xor_sync(0xFFFFFFFFu, sns, o);
        wide |= __shfl_xor_sync(0xFFFFFFFFu, wide, o);
    }
    if (lane == 0) {
        atomicAdd(&s_tb, (unsigned long long)tb);
        atomicAdd(&s_ns, (unsigned long long)ns);
        atomicAdd(&s_stb, (unsigned long long)stb);
        atomicAdd(&s_sns, (unsigned long long)sns);
        if (wide) s_wide = 1;
    }
    __syncthreads();
    if (tid == 0) {
        conf->total_tiles = s_carry;
        conf->r = enc_clamp_r<Sym>(r_override >= 0 ? r_override : enc_rule_r(s_tb, s_ns));
        conf->entry32 = s_wide ? 0u : 1u;
        conf->seg_total = seg_first ? s_scarry : 0u;
        conf->seg_r = r_override >= 0 ? r_override : enc_rule_r(s_stb, s_sns);
        conf->seg_long = s_slong;
        if (seg_first) seg_first[nfields] = s_scarry;
    }
}

template <typename Sym>
static huff_status plan_launch(EncField *d_fields, uint32_t nfields, EncBatchConf *d_conf, int r_override,
                               uint32_t nsub_cap, uint32_t *seg_first, cudaStream_t st) {
    batch_plan_kernel<Sym><<<1, kPlanThreads, 0, st>>>(d_fields, nfields, d_conf, r_override, nsub_cap, seg_first);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

static uint32_t pow2_at_least(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <typename Sym>
static void (*batch_encode_kernel(uint32_t max_nbins))(EncArgs) {
    return max_nbins > kEncSmemTableBins ? encode_kernel<Sym, true, true> : encode_kernel<Sym, false, true>;
}

template <typename Sym>
static huff_status prepare(uint32_t max_nbins, uint32_t nfields, int *ctas_per_sm) {
    const bool gtab = max_nbins > kEncSmemTableBins;
    const size_t smem = enc_smem_bytes<Sym>(gtab, pow2_at_least(max_nbins), nfields);
    auto kern = batch_encode_kernel<Sym>(max_nbins);
    if (!allow_dynamic_smem((const void *)kern, smem))
        return HUFF_ERR_CUDA;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kEncCtaThreads, smem);
    *ctas_per_sm = occ;
    return occ >= 1 ? HUFF_OK : HUFF_ERR_INVALID_ARG;
}

template <typename Sym>
static huff_status launch(const EncField *d_fields, uint32_t nfields, const EncBatchConf *d_conf,
                          uint32_t max_nbins, uint8_t *scratch, uint32_t grid, cudaStream_t st) {
    EncArgs a{};
    a.fields = d_fields;
    a.conf = d_conf;
    a.nfields = nfields;
    a.tslots = pow2_at_least(max_nbins);
    a.tile_counter = reinterpret_cast<uint32_t *>(scratch);
    a.desc = reinterpret_cast<uint64_t *>(scratch + 64);
    a.reduce_log2 = -1;
    a.nsub_cap = kEncMaxSubs;
    const bool gtab = max_nbins > kEncSmemTableBins;
    const size_t smem = enc_smem_bytes<Sym>(gtab, a.tslots, nfields);
    batch_encode_kernel<Sym>(max_nbins)<<<grid, kEncCtaThreads, smem, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

// Batched segment form: the 32-bit entries of every field the planner gave
// segment tiles (blockIdx.y = field).
__global__ void seg_entry_kernel(const EncField *fields, const uint32_t *seg_first) {
    const uint32_t f = blockIdx.y;
    if (seg_first[f + 1] == seg_first[f]) return;
    const EncField &F = fields[f];
    const uint64_t *gcw = reinterpret_cast<const uint64_t *>(F.book + cb_cw_offset());
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < F.nbins; i += gridDim.x * blockDim.x)
        F.etab[i] = seg_entry_from_cw(gcw[i]);
}

template <typename Sym>
static huff_status seg_prepare(uint32_t nfields) {
    return allow_dynamic_smem((const void *)encode_seg_batch_kernel<Sym>, seg_batch_smem_bytes<Sym>(nfields))
               ? HUFF_OK : HUFF_ERR_CUDA;
}

template <typename Sym>
static huff_status seg_launch(const EncField *d_fields, uint32_t nfields, const EncBatchConf *d_conf,
                              const uint32_t *seg_first, uint32_t max_nbins, uint8_t *scratch, uint32_t grid,
                              bool many, cudaStream_t st) {
    const uint32_t bx = std::min<uint32_t>(16u, (max_nbins + 255) / 256);
    seg_entry_kernel<<<dim3(bx, nfields), 256, 0, st>>>(d_fields, seg_first);
    note_launch();
    EncArgs a{};
    a.fields = d_fields;
    a.conf = d_conf;
    a.nfields = nfields;
    a.tslots = 1;
    a.tile_counter = reinterpret_cast<uint32_t *>(scratch);
    a.desc = reinterpret_cast<uint64_t *>(scratch + 64);
    a.reduce_log2 = -1;
    a.nsub_cap = kEncMaxSubs;
    a.seg_first = seg_first;
    a.seg_many = many ? 1u : 0u;
    encode_seg_batch_kernel<Sym><<<grid, kSegThreads, seg_batch_smem_bytes<Sym>(nfields), st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

uint32_t encode_seg_lane_symbols(huff_dtype dtype) {
    return dtype == HUFF_U8 ? seg_lane_syms<uint8_t>() : dtype == HUFF_U16 ? seg_lane_syms<uint16_t>()
                                                                             : seg_lane_syms<uint32_t>();
}

uint32_t encode_seg_tile_symbols(huff_dtype dtype) {
    return dtype == HUFF_U8 ? seg_sub_syms<uint8_t>() : dtype == HUFF_U16 ? seg_sub_syms<uint16_t>()
                                                                            : seg_sub_syms<uint32_t>();
}

huff_status encode_seg_batch_prepare(huff_dtype dtype, uint32_t nfields) {
    switch (dtype) {
        case HUFF_U8: return seg_prepare<uint8_t>(nfields);
        case HUFF_U16: return seg_prepare<uint16_t>(nfields);
        case HUFF_U32: return seg_prepare<uint32_t>(nfields);
    }
    return HUFF_ERR_INVALID_ARG;
}

huff_status encode_seg_batch_launch(huff_dtype dtype, const EncField *d_fields, uint32_t nfields,
                                    const EncBatchConf *d_conf, const uint32_t *seg_first, uint32_t max_nbins,
                                    uint8_t *scratch, uint32_t grid, bool many, cudaStream_t st) {
    switch (dtype) {
        case HUFF_U8: return seg_launch<uint8_t>(d_fields, nfields, d_conf, seg_first, max_nbins, scratch, grid, many, st);
        case HUFF_U16: return seg_launch<uint16_t>(d_fields, nfields, d_conf, seg_first, max_nbins, scratch, grid, many, st);
        case HUFF_U32: return seg_launch<uint32_t>(d_fields, nfields, d_conf, seg_first, max_nbins, scratch, grid, many, st);
    }
    return HUFF_ERR_INVALID_ARG;
}

huff_status encode_batch_prepare(huff_dtype dtype, uint32_t max_nbins, uint32_t nfields, int *ctas_per_sm) {
    switch (dtype) {
        case HUFF_U8: return prepare<uint8_t>(max_nbins, nfields, ctas_per_sm);
        case HUFF_U16: return prepare<uint16_t>(max_nbins, nfields, ctas_per_sm);
        case HUFF_U32: return prepare<uint32_t>(max_nbins, nfields, ctas_per_sm);
    }
    return HUFF_ERR_INVALID_ARG;
}

huff_status encode_batch_plan_launch(huff_dtype dtype, EncField *d_fields, uint32_t nfields, EncBatchConf *d_conf,
                                     int r_override, uint32_t nsub_cap, cudaStream_t st, uint32_t *seg_first) {
    switch (dtype) {
        case HUFF_U8: return plan_launch<uint8_t>(d_fields, nfields, d_conf, r_override, nsub_cap, seg_first, st);
        case HUFF_U16: return plan_launch<uint16_t>(d_fields, nfields, d_conf, r_override, nsub_cap, seg_first, st);
        case HUFF_U32: return plan_launch<uint32_t>(d_fields, nfields, d_conf, r_override, nsub_cap, seg_first, st);
    }
    return HUFF_ERR_INVALID_ARG;
}

huff_status encode_batch_launch(huff_dtype dtype, const EncField *d_fields, uint32_t nfields,
                                const EncBatchConf *d_conf, uint32_t max_nbins, uint8_t *scratch, uint32_t grid,
                                cudaStream_t st) {
    switch (dtype) {
        case HUFF_U8: return launch<uint8_t>(d_fields, nfields, d_conf, max_nbins, scratch, grid, st);
        case HUFF_U16: return launch<uint16_t>(d_fields, nfields, d_conf, max_nbins, scratch, grid, st);
        case HUFF_U32: return launch<uint32_t>(d_fields, nfields, d_conf, max_nbins, scratch, grid, st);
    }
    return HUFF_ERR_INVALID_ARG;
}

}  // namespace huff
