// Batched encoding plans (huff_batch_*): field grouping, the plan's device
// layout, capture of the launch set in a CUDA graph, and the autotuner that
// picks the encoder's reduction factor, tile size, CTAs per SM and (for
// fields that leave it open) chunk size by timing the graph on the fields.
// The encode stage takes one of three forms: one persistent launch of the
// general encoder whose tiles run over all fields of a group; one
// single-field launch per field (the segment encoder wherever the field's
// codewords allow it), fanned out over side streams inside the graph; or one
// persistent launch of the segment encoder over the fields whose codewords
// fit it, then the general encoder over the rest.  The tuner times all three.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.cuh"

namespace huff {

void launch_count_suppress(bool on);

constexpr uint32_t kGroupMaxFields = 512;     // encode keeps one first-tile id per field in shared memory
constexpr uint32_t kMaxBatchFields = 65536;
constexpr int kAutoChunkLog2[3] = {10, 12, 14};
#ifndef HUFF_BATCH_SIDE_STREAMS
#define HUFF_BATCH_SIDE_STREAMS 64
#endif
constexpr int kSideStreams = HUFF_BATCH_SIDE_STREAMS;   // per-field encode launches run on these, concurrently
constexpr int kPerFieldTiles[3] = {8, 16, 32};          // tuner: least tiles per CTA of a per-field launch

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static int alphabet_class(uint32_t nbins) { return nbins <= 4096 ? 0 : nbins <= 16384 ? 1 : 2; }

struct BatchGroup {
    huff_dtype dtype;
    uint32_t max_nbins;
    std::vector<uint32_t> idx;          // plan field ids
    std::vector<HistTile> tiles;
    std::vector<HistField> hfields;
    std::vector<CbArgs> cbargs;
    std::vector<EncField> efields;      // host copy (chunk sizes are set from it)
    size_t off_tiles = 0, off_hf = 0, off_cb = 0, off_ef = 0, off_conf = 0, off_escr = 0, off_cbscr = 0;
    size_t escr_bytes = 0, cbscr_stride = 0;
    uint32_t grid_h = 1, grid_c = 1;
    int enc_occ = 1;                    // encode CTAs per SM that fit
    size_t off_fscr = 0, fscr_bytes = 0;
    std::vector<size_t> fscr;           // per field: its single-field encode scratch, from off_fscr
    size_t off_sfirst = 0, off_sscr = 0, sscr_bytes = 0, off_etab = 0;   // batched segment form
    bool seg_many = false;              // some field's chunks are shorter than a segment
    std::vector<uint32_t> by_size;      // field positions, most symbols first
};

struct Setting {
    int r;              // -1 = rule
    int max_subtiles;
    int ctas_per_sm;    // 0 = as many as fit
    int chunk_log2;     // M for fields created with -1
    int per_field;      // k >= 1: one single-field encode launch per field, at least k tiles per CTA
    int seg;            // 1: the batched segment form (per_field 0)
};

}  // namespace huff

using namespace huff;

struct huff_batch_plan {
    int device = 0;
    std::vector<huff_field> fields;
    std::vector<int32_t> chunk_log2;    // M of each field in use
    std::vector<uint8_t> auto_chunk;    // field left M to the plan
    std::vector<BatchGroup> groups;
    std::vector<size_t> off_hist, off_book;
    size_t off_status = 0, off_hist0 = 0, hist_bytes = 0;
    uint8_t *dmem = nullptr;
    size_t dbytes = 0;
    cudaStream_t cs = nullptr;          // capture / tuning stream
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kSideStreams] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Setting cur{};
    uint32_t kernels_per_run = 0;
    uint32_t candidates = 0;
    float tuned_ms = 0.f;
};

namespace {

bool field_ok(const huff_field &f) {
    const huff_dtype d = f.dtype;
    if (d != HUFF_U8 && d != HUFF_U16 && d != HUFF_U32) return false;
    if (f.nbins < 1 || f.nbins > HUFF_MAX_BINS_BATCH || (d == HUFF_U8 && f.nbins > 256)) return false;
    if (f.n >= (1ull << 32)) return false;
    if (!f.d_chunk_bit_offset || !f.d_total_bits) return false;
    if (f.n && (!f.d_sym || !f.d_out)) return false;
    if (((uintptr_t)f.d_sym % (uintptr_t)d) != 0 || ((uintptr_t)f.d_out & 3) != 0 ||
        ((uintptr_t)f.d_chunk_bit_offset & 7) != 0 || ((uintptr_t)f.d_total_bits & 7) != 0)
        return false;
    if (f.chunk_log2 != -1 && (f.chunk_log2 < 4 || f.chunk_log2 > 30 || f.chunk_log2 < encode_run_log2(d)))
        return false;
    return true;
}

uint32_t *status_ptr(huff_batch_plan *p, uint32_t i) {
    return reinterpret_cast<uint32_t *>(p->dmem + p->off_status) + i;
}

// Fills the chunk-size dependent members of every encode record for setting s
// and uploads them.
huff_status apply_chunks(huff_batch_plan *p, int auto_m) {
    for (uint32_t i = 0; i < p->fields.size(); i++)
        p->chunk_log2[i] = p->auto_chunk[i] ? auto_m : p->fields[i].chunk_log2;
    for (BatchGroup &g : p->groups) {
        g.seg_many = false;
        for (size_t k = 0; k < g.idx.size(); k++) {
            EncField &e = g.efields[k];
            const int m = p->chunk_log2[g.idx[k]];
            e.chunk_log2 = m;
            e.nchunks = (e.n + (1ull << m) - 1) >> m;
            if ((1ull << m) < encode_seg_lane_symbols(g.dtype)) g.seg_many = true;
        }
        if (cudaMemcpyAsync(p->dmem + g.off_ef, g.efields.data(), g.efields.size() * sizeof(EncField),
                            cudaMemcpyHostToDevice, p->cs) != cudaSuccess)
            return HUFF_ERR_CUDA;
    }
    return cudaStreamSynchronize(p->cs) == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

// The encode stage as one single-field launch per field (its scratch cleared
// already): fanned out from st over the side streams, each field to the
// stream with the fewest symbols so far (largest fields first), and joined
// back into st.
huff_status encode_fields(huff_batch_plan *p, const BatchGroup &g, const Setting &s, cudaStream_t st) {
    const int ns = (int)std::min<size_t>(kSideStreams, g.idx.size());
    if (cudaEventRecord(p->fork, st) != cudaSuccess) return HUFF_ERR_CUDA;
    for (int k = 0; k < ns; k++)
        if (cudaStreamWaitEvent(p->side[k], p->fork, 0) != cudaSuccess) return HUFF_ERR_CUDA;
    uint64_t load[kSideStreams] = {};
    for (uint32_t fi : g.by_size) {
        int k = 0;
        for (int j = 1; j < ns; j++)
            if (load[j] < load[k]) k = j;
        const uint32_t i = g.idx[fi];
        const huff_field &f = p->fields[i];
        load[k] += f.n + 1;
        if (f.n == 0) {
            if (cudaMemsetAsync(f.d_chunk_bit_offset, 0, 8, p->side[k]) != cudaSuccess ||
                cudaMemsetAsync(f.d_total_bits, 0, 8, p->side[k]) != cudaSuccess)
                return HUFF_ERR_CUDA;
            continue;
        }
        const huff_status e = encode_launch_ex(f.d_sym, f.n, f.dtype, p->dmem + p->off_book[i], f.nbins,
                                               p->chunk_log2[i], s.r, 0u, static_cast<uint32_t *>(f.d_out),
                                               f.out_capacity_words, f.d_chunk_bit_offset, f.d_total_bits,
                                               p->dmem + g.off_fscr + g.fscr[fi], status_ptr(p, i), p->side[k], 0u,
                                               0u, true, (uint32_t)s.per_field, true);
        if (e != HUFF_OK) return e;
    }
    for (int k = 0; k < ns; k++) {
        if (cudaEventRecord(p->join[k], p->side[k]) != cudaSuccess) return HUFF_ERR_CUDA;
        if (cudaStreamWaitEvent(st, p->join[k], 0) != cudaSuccess) return HUFF_ERR_CUDA;
    }
    return HUFF_OK;
}

// The launch set of one batch run, enqueued on st (captured into the graph).
// With ev (5 events per group), events are recorded around each stage.
huff_status record(huff_batch_plan *p, const Setting &s, cudaStream_t st, const cudaEvent_t *ev = nullptr) {
    if (cudaMemsetAsync(p->dmem + p->off_status, 0, 4 * p->fields.size(), st) != cudaSuccess) return HUFF_ERR_CUDA;
    if (p->hist_bytes && cudaMemsetAsync(p->dmem + p->off_hist0, 0, p->hist_bytes, st) != cudaSuccess)
        return HUFF_ERR_CUDA;
    const int sms = sm_count();
    int gi = 0;
    auto mark = [&](int k) { return ev ? cudaEventRecord(ev[5 * gi + k], st) == cudaSuccess : true; };
    for (BatchGroup &g : p->groups) {
        const uint32_t nf = (uint32_t)g.idx.size();
        huff_status e;
        if (!mark(0)) return HUFF_ERR_CUDA;
        if (!g.tiles.empty()) {
            e = histogram_batch_launch(g.dtype, reinterpret_cast<const HistTile *>(p->dmem + g.off_tiles),
                                       (uint32_t)g.tiles.size(),
                                       reinterpret_cast<const HistField *>(p->dmem + g.off_hf), g.max_nbins,
                                       g.grid_h, st);
            if (e != HUFF_OK) return e;
        }
        if (!mark(1)) return HUFF_ERR_CUDA;
        e = codebook_batch_launch(reinterpret_cast<const CbArgs *>(p->dmem + g.off_cb), nf, g.max_nbins, g.grid_c,
                                  g.cbscr_stride ? p->dmem + g.off_cbscr : nullptr, g.cbscr_stride, st);
        if (e != HUFF_OK) return e;
        if (s.seg) {
            EncField *ef = reinterpret_cast<EncField *>(p->dmem + g.off_ef);
            EncBatchConf *conf = reinterpret_cast<EncBatchConf *>(p->dmem + g.off_conf);
            uint32_t *sfirst = reinterpret_cast<uint32_t *>(p->dmem + g.off_sfirst);
            if (!mark(2)) return HUFF_ERR_CUDA;
            e = encode_batch_plan_launch(g.dtype, ef, nf, conf, s.r, (uint32_t)s.max_subtiles, st, sfirst);
            if (e != HUFF_OK) return e;
            if (cudaMemsetAsync(p->dmem + g.off_escr, 0, g.escr_bytes, st) != cudaSuccess ||
                cudaMemsetAsync(p->dmem + g.off_sscr, 0, g.sscr_bytes, st) != cudaSuccess)
                return HUFF_ERR_CUDA;
            if (!mark(3)) return HUFF_ERR_CUDA;
            e = encode_seg_batch_launch(g.dtype, ef, nf, conf, sfirst, g.max_nbins, p->dmem + g.off_sscr,
                                        (uint32_t)(sms * 2), g.seg_many, st);
            if (e != HUFF_OK) return e;
            int c = s.ctas_per_sm <= 0 ? g.enc_occ : std::min(s.ctas_per_sm, g.enc_occ);
            if (c < 1) c = 1;
            e = encode_batch_launch(g.dtype, ef, nf, conf, g.max_nbins, p->dmem + g.off_escr, (uint32_t)(sms * c), st);
            if (e != HUFF_OK) return e;
            if (!mark(4)) return HUFF_ERR_CUDA;
            gi++;
            continue;
        }
        if (s.per_field) {
            if (!mark(2)) return HUFF_ERR_CUDA;
            if (cudaMemsetAsync(p->dmem + g.off_fscr, 0, g.fscr_bytes, st) != cudaSuccess) return HUFF_ERR_CUDA;
            if (!mark(3)) return HUFF_ERR_CUDA;
            if ((e = encode_fields(p, g, s, st)) != HUFF_OK) return e;
            if (!mark(4)) return HUFF_ERR_CUDA;
            gi++;
            continue;
        }
        EncField *ef = reinterpret_cast<EncField *>(p->dmem + g.off_ef);
        EncBatchConf *conf = reinterpret_cast<EncBatchConf *>(p->dmem + g.off_conf);
        if (!mark(2)) return HUFF_ERR_CUDA;
        e = encode_batch_plan_launch(g.dtype, ef, nf, conf, s.r, (uint32_t)s.max_subtiles, st);
        if (e != HUFF_OK) return e;
        if (cudaMemsetAsync(p->dmem + g.off_escr, 0, g.escr_bytes, st) != cudaSuccess) return HUFF_ERR_CUDA;
        int c = s.ctas_per_sm <= 0 ? g.enc_occ : std::min(s.ctas_per_sm, g.enc_occ);
        if (c < 1) c = 1;
        if (!mark(3)) return HUFF_ERR_CUDA;
        e = encode_batch_launch(g.dtype, ef, nf, conf, g.max_nbins, p->dmem + g.off_escr, (uint32_t)(sms * c), st);
        if (e != HUFF_OK) return e;
        if (!mark(4)) return HUFF_ERR_CUDA;
        gi++;
    }
    return HUFF_OK;
}

// Kernel launches of one run in the plan's current setting.
uint32_t count_kernels(const huff_batch_plan *p) {
    uint32_t k = 0;
    for (const BatchGroup &g : p->groups) {
        k += (g.tiles.empty() ? 0 : 1) + 1;                 // histogram, codebooks
        if (p->cur.seg) {
            k += 4;                                          // planner, entry tables, both encoders
            continue;
        }
        if (!p->cur.per_field) {
            k += 2;                                          // tile planner, encode
            continue;
        }
        for (uint32_t i : g.idx)
            if (p->fields[i].n) k += encode_kernels_per_call(p->fields[i].nbins);
    }
    return k;
}

void drop_graph(huff_batch_plan *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

huff_status capture(huff_batch_plan *p, const Setting &s) {
    drop_graph(p);
    if (cudaStreamBeginCapture(p->cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HUFF_ERR_CUDA;
    launch_count_suppress(true);
    huff_status e = record(p, s, p->cs);
    launch_count_suppress(false);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(p->cs, &g);
    if (e != HUFF_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e != HUFF_OK ? e : HUFF_ERR_CUDA;
    }
    p->graph = g;
    if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
        drop_graph(p);
        return HUFF_ERR_CUDA;
    }
    return HUFF_OK;
}

// Best of `reps` timed runs of the current graph (after one untimed run), in ms.
huff_status time_graph(huff_batch_plan *p, int reps, float *best) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return HUFF_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HUFF_ERR_CUDA;
    }
    huff_status st = HUFF_OK;
    float b = 1e30f;
    if (cudaGraphLaunch(p->exec, p->cs) != cudaSuccess) st = HUFF_ERR_CUDA;
    for (int r = 0; r < reps && st == HUFF_OK; r++) {
        float ms = 0.f;
        if (cudaEventRecord(e0, p->cs) != cudaSuccess || cudaGraphLaunch(p->exec, p->cs) != cudaSuccess ||
            cudaEventRecord(e1, p->cs) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = HUFF_ERR_CUDA;
            break;
        }
        b = std::min(b, ms);
    }
    if (cudaStreamSynchronize(p->cs) != cudaSuccess) st = HUFF_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best = b;
    return st;
}

huff_status autotune(huff_batch_plan *p) {
    int rmin = 4, rmax = 0, occ = 1;
    for (const BatchGroup &g : p->groups) {
        int a, b;
        encode_r_range(g.dtype, &a, &b);
        rmin = std::min(rmin, a);
        rmax = std::max(rmax, b);
        occ = std::max(occ, g.enc_occ);
    }
    const bool any_auto = std::find(p->auto_chunk.begin(), p->auto_chunk.end(), 1) != p->auto_chunk.end();
    std::vector<int> ms_list = any_auto ? std::vector<int>(kAutoChunkLog2, kAutoChunkLog2 + 3) : std::vector<int>{0};
    Setting best{-1, 8, 0, any_auto ? 10 : 0, 0, 0};
    float best_ms = 1e30f;
    uint32_t count = 0;
    huff_status e0 = apply_chunks(p, 10);
    if (e0 != HUFF_OK) return e0;
    for (int r = rmin; r <= rmax; r++)
        for (int cap : {2, 4, 8})
            for (int c = 1; c <= std::min(occ, 3); c++) {
                Setting s{r, cap, c, 0, 0, 0};
                huff_status e = capture(p, s);
                if (e != HUFF_OK) return e;
                for (int m : ms_list) {
                    if (any_auto && (e = apply_chunks(p, m)) != HUFF_OK) return e;
                    float t;
                    if ((e = time_graph(p, 3, &t)) != HUFF_OK) return e;
                    count++;
                    if (t < best_ms) {
                        best_ms = t;
                        best = s;
                        best.chunk_log2 = m;
                    }
                }
            }
    // one launch per field (r by rule: on the segment path r moves the time little)
    // the batched segment form (r by rule over its fields; the rest keeps the
    // general encoder at 8 sub-tiles and the CTAs that fit), then one launch
    // per field
    for (int per : {0, kPerFieldTiles[0], kPerFieldTiles[1], kPerFieldTiles[2]}) {
        const Setting s{-1, 8, 0, 0, per, per == 0 ? 1 : 0};
        huff_status e = capture(p, s);
        if (e != HUFF_OK) return e;
        for (int m : ms_list) {
            if (any_auto && (e = apply_chunks(p, m)) != HUFF_OK) return e;
            float t;
            if ((e = time_graph(p, 3, &t)) != HUFF_OK) return e;
            count++;
            if (t < best_ms) {
                best_ms = t;
                best = s;
                best.chunk_log2 = m;
            }
        }
    }
    p->candidates = count;
    p->tuned_ms = best_ms;
    p->cur = best;
    if (any_auto) {
        huff_status e = apply_chunks(p, best.chunk_log2);
        if (e != HUFF_OK) return e;
    }
    return capture(p, best);
}

void free_plan(huff_batch_plan *p) {
    if (!p) return;
    if (p->cs) cudaStreamSynchronize(p->cs);
    for (cudaStream_t s : p->side)
        if (s) cudaStreamSynchronize(s);
    drop_graph(p);
    if (p->dmem) cudaFree(p->dmem);
    if (p->cs) cudaStreamDestroy(p->cs);
    for (cudaStream_t s : p->side)
        if (s) cudaStreamDestroy(s);
    if (p->fork) cudaEventDestroy(p->fork);
    for (cudaEvent_t e : p->join)
        if (e) cudaEventDestroy(e);
    delete p;
}

}  // namespace

extern "C" {

void huff_batch_default_cfg(huff_batch_cfg *cfg) {
    if (!cfg) return;
    cfg->autotune = 0;
    cfg->reduce_log2 = -1;
    cfg->max_subtiles = 0;
    cfg->ctas_per_sm = 0;
    cfg->encode_form = 0;
}

huff_status huff_batch_plan_create(const huff_field *fields, uint32_t nfields, const huff_batch_cfg *cfg,
                                   void *stream, huff_batch_plan **out) {
    if (!out) return HUFF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!fields || nfields < 1 || nfields > kMaxBatchFields) return HUFF_ERR_INVALID_ARG;
    huff_batch_cfg c;
    huff_batch_default_cfg(&c);
    if (cfg) c = *cfg;
    if (c.reduce_log2 < -1 || c.reduce_log2 > 4 || c.max_subtiles < 0 || c.max_subtiles > 8 || c.ctas_per_sm < 0 ||
        c.encode_form < 0 || c.encode_form > 2)
        return HUFF_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < nfields; i++)
        if (!field_ok(fields[i])) return HUFF_ERR_INVALID_ARG;

    huff_batch_plan *p = new (std::nothrow) huff_batch_plan();
    if (!p) return HUFF_ERR_OOM;
    cudaGetDevice(&p->device);
    p->fields.assign(fields, fields + nfields);
    p->chunk_log2.assign(nfields, 10);
    p->auto_chunk.assign(nfields, 0);
    for (uint32_t i = 0; i < nfields; i++) p->auto_chunk[i] = fields[i].chunk_log2 == -1;

    // ---- groups: by dtype and alphabet class, at most kGroupMaxFields each
    std::vector<uint32_t> order(nfields);
    for (uint32_t i = 0; i < nfields; i++) order[i] = i;
    auto key = [&](uint32_t i) { return (int)fields[i].dtype * 4 + alphabet_class(fields[i].nbins); };
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return key(a) < key(b); });
    for (uint32_t k = 0; k < nfields;) {
        BatchGroup g;
        g.dtype = fields[order[k]].dtype;
        const int kk = key(order[k]);
        while (k < nfields && key(order[k]) == kk && g.idx.size() < kGroupMaxFields) g.idx.push_back(order[k++]);
        g.max_nbins = 1;
        for (uint32_t i : g.idx) g.max_nbins = std::max(g.max_nbins, fields[i].nbins);
        p->groups.push_back(std::move(g));
    }

    // ---- device layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = align_up(off, 256);
        const size_t at = off;
        off += bytes;
        return at;
    };
    p->off_status = take(4ull * nfields);
    p->off_hist.resize(nfields);
    p->off_book.resize(nfields);
    off = align_up(off, 256);
    p->off_hist0 = off;
    for (uint32_t i = 0; i < nfields; i++) {
        p->off_hist[i] = off;
        off += align_up(4ull * fields[i].nbins, 16);
    }
    p->hist_bytes = off - p->off_hist0;
    for (uint32_t i = 0; i < nfields; i++) p->off_book[i] = take(align_up(huff_codebook_bytes(fields[i].nbins), 16));
    const int sms = sm_count();
    for (BatchGroup &g : p->groups) {
        const uint64_t ht = histogram_batch_tile(g.max_nbins);
        const uint32_t sub = encode_sub_symbols(g.dtype);
        uint64_t max_tiles = 0;
        for (uint32_t fi = 0; fi < g.idx.size(); fi++) {
            const huff_field &f = fields[g.idx[fi]];
            for (uint64_t s0 = 0; s0 < f.n; s0 += ht) g.tiles.push_back(HistTile{fi, 0, s0, std::min(f.n, s0 + ht)});
            max_tiles += (f.n + sub - 1) / sub;
        }
        g.off_tiles = take(sizeof(HistTile) * std::max<size_t>(1, g.tiles.size()));
        g.off_hf = take(sizeof(HistField) * g.idx.size());
        g.off_cb = take(sizeof(CbArgs) * g.idx.size());
        g.off_ef = take(sizeof(EncField) * g.idx.size());
        g.off_conf = take(sizeof(EncBatchConf));
        g.escr_bytes = 64 + 16 * max_tiles;
        g.off_escr = take(g.escr_bytes);
        size_t fs = 0;
        for (uint32_t fi = 0; fi < g.idx.size(); fi++) {
            const huff_field &f = fields[g.idx[fi]];
            g.fscr.push_back(fs);
            fs += align_up(encode_scratch_bytes(f.n, f.nbins), 256);
        }
        g.fscr_bytes = std::max<size_t>(fs, 256);
        g.off_fscr = take(g.fscr_bytes);
        // batched segment form: first tile ids, descriptors, entry tables
        uint64_t seg_tiles = 0;
        const uint32_t seg_sub = encode_seg_tile_symbols(g.dtype);
        for (uint32_t i : g.idx) seg_tiles += (fields[i].n + seg_sub - 1) / seg_sub;
        g.off_sfirst = take(4ull * (g.idx.size() + 1));
        g.sscr_bytes = 64 + 16 * seg_tiles;
        g.off_sscr = take(g.sscr_bytes);
        size_t et = 0;
        for (uint32_t i : g.idx) et += align_up(4ull * fields[i].nbins, 16);
        g.off_etab = take(std::max<size_t>(et, 16));
        g.by_size.resize(g.idx.size());
        for (uint32_t fi = 0; fi < g.idx.size(); fi++) g.by_size[fi] = fi;
        std::stable_sort(g.by_size.begin(), g.by_size.end(),
                         [&](uint32_t a, uint32_t b) { return fields[g.idx[a]].n > fields[g.idx[b]].n; });
        // launch shapes (attributes are set here, before any capture)
        int occ_h = 1, occ_c = 1;
        huff_status e = histogram_batch_prepare(g.dtype, g.max_nbins, &occ_h);
        if (e == HUFF_OK) e = codebook_batch_prepare(g.max_nbins, &occ_c);
        if (e == HUFF_OK) e = encode_batch_prepare(g.dtype, g.max_nbins, (uint32_t)g.idx.size(), &g.enc_occ);
        if (e == HUFF_OK) e = encode_seg_batch_prepare(g.dtype, (uint32_t)g.idx.size());
        for (uint32_t fi = 0; fi < g.idx.size() && e == HUFF_OK; fi++)
            e = encode_prepare(g.dtype, fields[g.idx[fi]].nbins);
        if (e != HUFF_OK) {
            free_plan(p);
            return e;
        }
        g.grid_h = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sms * occ_h, g.tiles.size()));
        g.grid_c = (uint32_t)std::min<uint64_t>((uint64_t)sms * occ_c, g.idx.size());
        if (g.max_nbins > 4096) {
            g.cbscr_stride = align_up(codebook_array_bytes(g.max_nbins), 256);
            g.off_cbscr = take(g.cbscr_stride * g.grid_c);
        }
    }
    p->dbytes = align_up(off, 256);
    if (cudaMalloc(&p->dmem, p->dbytes) != cudaSuccess) {
        p->dmem = nullptr;
        free_plan(p);
        return HUFF_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking) != cudaSuccess) {
        p->cs = nullptr;
        free_plan(p);
        return HUFF_ERR_CUDA;
    }
    bool made = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) == cudaSuccess;
    if (!made) p->fork = nullptr;
    for (int k = 0; k < kSideStreams && made; k++) {
        if (cudaStreamCreateWithFlags(&p->side[k], cudaStreamNonBlocking) != cudaSuccess) {
            p->side[k] = nullptr;
            made = false;
        } else if (cudaEventCreateWithFlags(&p->join[k], cudaEventDisableTiming) != cudaSuccess) {
            p->join[k] = nullptr;
            made = false;
        }
    }
    if (!made) {
        free_plan(p);
        return HUFF_ERR_CUDA;
    }
    // the caller's stream may still be producing the fields' inputs
    if (stream && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        free_plan(p);
        return HUFF_ERR_CUDA;
    }

    // ---- records
    for (BatchGroup &g : p->groups) {
        size_t et = 0;
        for (uint32_t fi = 0; fi < g.idx.size(); fi++) {
            const uint32_t i = g.idx[fi];
            const huff_field &f = fields[i];
            uint32_t *hist = reinterpret_cast<uint32_t *>(p->dmem + p->off_hist[i]);
            uint8_t *book = p->dmem + p->off_book[i];
            const uintptr_t mis = (16 - ((uintptr_t)f.d_sym & 15)) & 15;
            g.hfields.push_back(HistField{static_cast<const uint8_t *>(f.d_sym), hist, status_ptr(p, i), f.nbins,
                                          (uint32_t)(mis / (uintptr_t)f.dtype)});
            g.cbargs.push_back(CbArgs{hist, f.nbins, book, nullptr, status_ptr(p, i)});
            EncField e{};
            e.sym = static_cast<const uint8_t *>(f.d_sym);
            e.book = book;
            e.out = f.d_out;
            e.offs = f.d_chunk_bit_offset;
            e.total_bits = f.d_total_bits;
            e.status = status_ptr(p, i);
            e.n = f.n;
            e.cap_words = f.out_capacity_words;
            e.nbins = f.nbins;
            e.aligned = ((uintptr_t)f.d_sym & 15) == 0;
            e.etab = reinterpret_cast<uint32_t *>(p->dmem + g.off_etab + et);
            et += align_up(4ull * f.nbins, 16);
            g.efields.push_back(e);
        }
        cudaError_t ce = cudaSuccess;
        if (!g.tiles.empty())
            ce = cudaMemcpyAsync(p->dmem + g.off_tiles, g.tiles.data(), g.tiles.size() * sizeof(HistTile),
                                 cudaMemcpyHostToDevice, p->cs);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(p->dmem + g.off_hf, g.hfields.data(), g.hfields.size() * sizeof(HistField),
                                 cudaMemcpyHostToDevice, p->cs);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(p->dmem + g.off_cb, g.cbargs.data(), g.cbargs.size() * sizeof(CbArgs),
                                 cudaMemcpyHostToDevice, p->cs);
        if (ce != cudaSuccess) {
            free_plan(p);
            return HUFF_ERR_CUDA;
        }
    }
    huff_status e;
    if (c.autotune) {
        e = autotune(p);
    } else {
        p->cur = Setting{c.reduce_log2, c.max_subtiles ? c.max_subtiles : 8, c.ctas_per_sm, 10,
                         c.encode_form == 1 ? 16 : 0, c.encode_form == 2 ? 1 : 0};
        e = apply_chunks(p, 10);
        if (e == HUFF_OK) e = capture(p, p->cur);
    }
    if (e == HUFF_OK && cudaStreamSynchronize(p->cs) != cudaSuccess) e = HUFF_ERR_CUDA;
    if (e != HUFF_OK) {
        free_plan(p);
        return e;
    }
    p->kernels_per_run = count_kernels(p);
    *out = p;
    return HUFF_OK;
}

huff_status huff_batch_encode(huff_batch_plan *p, void *stream) {
    if (!p || !p->exec) return HUFF_ERR_INVALID_ARG;
    if (cudaGraphLaunch(p->exec, (cudaStream_t)stream) != cudaSuccess) return HUFF_ERR_CUDA;
    note_launch((int)p->kernels_per_run);
    return HUFF_OK;
}

huff_status huff_batch_profile(huff_batch_plan *p, void *stream, float *stage_ms) {
    if (!p || !stage_ms) return HUFF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<cudaEvent_t> ev(5 * p->groups.size(), nullptr);
    huff_status e = HUFF_OK;
    for (auto &x : ev)
        if (cudaEventCreate(&x) != cudaSuccess) { x = nullptr; e = HUFF_ERR_CUDA; }
    if (e == HUFF_OK) e = record(p, p->cur, st, ev.data());
    if (e == HUFF_OK && cudaStreamSynchronize(st) != cudaSuccess) e = HUFF_ERR_CUDA;
    for (int k = 0; k < 4; k++) stage_ms[k] = 0.f;
    for (size_t g = 0; g < p->groups.size() && e == HUFF_OK; g++)
        for (int k = 0; k < 4; k++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[5 * g + k], ev[5 * g + k + 1]) != cudaSuccess) {
                e = HUFF_ERR_CUDA;
                break;
            }
            stage_ms[k] += ms;
        }
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    return e;
}

huff_status huff_batch_status(huff_batch_plan *p, uint32_t *h_status, void *stream) {
    if (!p || !h_status) return HUFF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(h_status, p->dmem + p->off_status, 4 * p->fields.size(), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return HUFF_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

huff_status huff_batch_get_info(const huff_batch_plan *p, huff_batch_info *info) {
    if (!p || !info) return HUFF_ERR_INVALID_ARG;
    info->reduce_log2 = p->cur.r;
    info->max_subtiles = p->cur.max_subtiles;
    info->ctas_per_sm = p->cur.ctas_per_sm;
    const bool any_auto = std::find(p->auto_chunk.begin(), p->auto_chunk.end(), 1) != p->auto_chunk.end();
    info->chunk_log2 = any_auto ? p->cur.chunk_log2 : 0;
    info->groups = (uint32_t)p->groups.size();
    info->kernels_per_run = p->kernels_per_run;
    info->candidates = p->candidates;
    info->tuned_ms = p->tuned_ms;
    info->device_bytes = p->dbytes;
    info->encode_form = p->cur.seg ? 2u : p->cur.per_field ? 1u : 0u;
    info->per_field_tiles = (uint32_t)p->cur.per_field;
    return HUFF_OK;
}

const void *huff_batch_codebook(const huff_batch_plan *p, uint32_t field) {
    if (!p || field >= p->fields.size()) return nullptr;
    return p->dmem + p->off_book[field];
}

const uint32_t *huff_batch_histogram(const huff_batch_plan *p, uint32_t field) {
    if (!p || field >= p->fields.size()) return nullptr;
    return reinterpret_cast<const uint32_t *>(p->dmem + p->off_hist[field]);
}

int huff_batch_chunk_log2(const huff_batch_plan *p, uint32_t field) {
    if (!p || field >= p->fields.size()) return -1;
    return p->chunk_log2[field];
}

void huff_batch_plan_destroy(huff_batch_plan *p) { free_plan(p); }

}  // extern "C"
