// Served form (huff_serve_*): jobs are admitted in arrival order against a
// device memory budget (RegionAllocator over one allocation), launched as
// batches of the batched kernels on a set of stream contexts as soon as a
// context is free (continuous batching: jobs that arrive while batches run
// join the next batch, which overlaps with the running ones), and completed
// by a host function queued behind each batch.  All bookkeeping is host C++;
// every step of the encoding runs in the library's kernels.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"
#include "pool.h"

namespace huff {
namespace {

constexpr uint32_t kMaxGroupsPerBatch = 16;
constexpr uint32_t kCbScratchCtas = 16;      // codebook CTAs of a large-alphabet group (each needs scratch)

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int alphabet_class(uint32_t nbins) { return nbins <= 4096 ? 0 : nbins <= 16384 ? 1 : 2; }

// Output words that always suffice: a Huffman code is never longer on
// average than the fixed-length code of ceil(log2 nbins) bits.
uint64_t result_words(uint64_t n, uint32_t nbins) {
    uint32_t b = 0;
    while ((1ull << b) < nbins) b++;
    if (b == 0) b = 1;
    return (n * b + 31) / 32 + 1;
}

enum class JobState { Queued, Admitted, Launched, Done };

struct Job {
    huff_request rq{};
    JobState state = JobState::Queued;
    bool release_when_done = false;
    bool holds_slot = false;             // admitted: counts against max_inflight until released
    uint64_t pool_off = 0, pool_bytes = 0;
    uint32_t *d_out = nullptr;
    uint64_t cap_words = 0;
    uint64_t *d_offs = nullptr;
    uint8_t *d_book = nullptr;
    huff_status status = HUFF_OK;
    uint64_t total_bits = 0;
    double t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
};

struct Ctx {
    huff_server *srv = nullptr;
    cudaStream_t st = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;       // jobs of the batch on the device (record k = tickets[k])
    uint8_t *dmem = nullptr;
    uint8_t *hmem = nullptr;
    HistTile *d_tiles = nullptr, *h_tiles = nullptr;
    HistField *d_hf = nullptr, *h_hf = nullptr;
    CbArgs *d_cb = nullptr, *h_cb = nullptr;
    EncField *d_ef = nullptr, *h_ef = nullptr;
    EncBatchConf *d_conf = nullptr;
    uint32_t *d_hist = nullptr;
    uint32_t *d_status = nullptr, *h_status = nullptr;
    uint64_t *d_total = nullptr, *h_total = nullptr;
    uint8_t *d_escr = nullptr, *d_cbscr = nullptr;
    size_t escr_bytes = 0;
    size_t cbscr_stride = 0;
    uint64_t max_tiles = 0;
};

}  // namespace
}  // namespace huff

using namespace huff;

struct huff_server {
    huff_serve_cfg cfg{};
    int device = 0;
    int sms = 1;
    uint8_t *pool_base = nullptr;
    RegionAllocator pool;
    std::mutex mu;
    std::condition_variable cv;          // dispatcher wake-ups
    std::condition_variable cv_done;     // job completions
    std::deque<uint64_t> queue;          // submitted, waiting for admission
    std::deque<uint64_t> admitted;       // admitted, waiting for a stream context
    std::unordered_map<uint64_t, Job> jobs;
    uint64_t next_ticket = 1;
    std::vector<Ctx> ctxs;
    std::thread dispatcher;
    bool stop = false;
    uint32_t inflight = 0;               // admitted and not released
    uint32_t running = 0;                // batches on the device
    huff_serve_stats stats{};
};

namespace {

uint64_t job_bytes(const huff_server *s, const huff_request &r) {
    const int m = s->cfg.chunk_log2;
    const uint64_t nch = (r.n + (1ull << m) - 1) >> m;
    return align256(4 * result_words(r.n, r.nbins)) + align256(8 * (nch + 1)) + align256(huff_codebook_bytes(r.nbins));
}

void free_job_memory(huff_server *s, Job &j) {
    if (j.pool_bytes) s->pool.release(j.pool_off, j.pool_bytes);
    j.pool_bytes = 0;
}

// Finishes a job (lock held): records its result, frees it if released.
void finish_locked(huff_server *s, uint64_t ticket, huff_status st, uint64_t total_bits, double t) {
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return;
    Job &j = it->second;
    j.status = st;
    j.total_bits = total_bits;
    j.t_done = t;
    j.state = JobState::Done;
    if (st == HUFF_ERR_CANCELLED) s->stats.cancelled++;
    else {
        s->stats.completed++;
        s->stats.symbols_done += j.rq.n;
    }
    if (j.release_when_done) {
        free_job_memory(s, j);
        if (j.holds_slot) s->inflight--;
        s->jobs.erase(it);
    }
}

void CUDART_CB batch_done(void *user) {
    Ctx *c = static_cast<Ctx *>(user);
    huff_server *s = c->srv;
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (size_t k = 0; k < c->tickets.size(); k++)
            finish_locked(s, c->tickets[k], (huff_status)c->h_status[k], c->h_total[k], t);
        c->tickets.clear();
        c->busy = false;
        s->running--;
        s->stats.pool_used = s->pool.used();
    }
    s->cv.notify_all();
    s->cv_done.notify_all();
}

void admit_locked(huff_server *s) {
    while (!s->queue.empty() && s->inflight < s->cfg.max_inflight) {
        Job &j = s->jobs[s->queue.front()];
        uint64_t off = 0;
        const uint64_t bytes = job_bytes(s, j.rq);
        if (!s->pool.alloc(bytes, &off)) break;         // arrival order: the head waits for memory
        j.pool_off = off;
        j.pool_bytes = bytes;
        const int m = s->cfg.chunk_log2;
        const uint64_t nch = (j.rq.n + (1ull << m) - 1) >> m;
        uint8_t *p = s->pool_base + off;
        j.cap_words = result_words(j.rq.n, j.rq.nbins);
        j.d_out = reinterpret_cast<uint32_t *>(p);
        p += align256(4 * j.cap_words);
        j.d_offs = reinterpret_cast<uint64_t *>(p);
        p += align256(8 * (nch + 1));
        j.d_book = p;
        j.state = JobState::Admitted;
        j.holds_slot = true;
        j.t_admit = now_s();
        s->inflight++;
        s->admitted.push_back(s->queue.front());
        s->queue.pop_front();
    }
    s->stats.pool_used = s->pool.used();
    s->stats.pool_peak = s->pool.peak();
}

struct GroupPlan {
    huff_dtype dtype;
    uint32_t max_nbins;
    uint32_t first, count;           // records [first, first + count)
    uint32_t tile_first, ntiles;
    uint64_t enc_tiles;              // descriptor bound of the group's encode
};

// Enqueues one batch on the context's stream (no lock held).  The batch's
// jobs (jb, with tickets tk) become records sorted by launch group (dtype and
// alphabet class); c->tickets[k] is the ticket of record k.
huff_status launch_batch(huff_server *s, Ctx *c, const std::vector<Job *> &jb0, const std::vector<uint64_t> &tk) {
    const uint32_t nj = (uint32_t)jb0.size();
    auto key = [](const Job *j) { return (int)j->rq.dtype * 4 + alphabet_class(j->rq.nbins); };
    std::vector<uint32_t> order(nj);
    for (uint32_t k = 0; k < nj; k++) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return key(jb0[a]) < key(jb0[b]); });
    std::vector<Job *> jb(nj);
    c->tickets.resize(nj);
    for (uint32_t k = 0; k < nj; k++) {
        jb[k] = jb0[order[k]];
        c->tickets[k] = tk[order[k]];
    }

    std::vector<GroupPlan> groups;
    uint64_t hist_words = 0;
    uint32_t ntiles = 0;
    for (uint32_t k = 0; k < nj;) {
        GroupPlan g{jb[k]->rq.dtype, 1, k, 0, ntiles, 0, 0};
        uint32_t e = k;
        while (e < nj && key(jb[e]) == key(jb[k])) {
            g.max_nbins = std::max(g.max_nbins, jb[e]->rq.nbins);
            e++;
        }
        g.count = e - k;
        const uint64_t ht = histogram_batch_tile(g.max_nbins);
        const uint32_t sub = encode_sub_symbols(g.dtype);
        for (uint32_t q = k; q < e; q++) {
            Job &j = *jb[q];
            const huff_request &r = j.rq;
            const uint32_t rec = q;
            for (uint64_t s0 = 0; s0 < r.n; s0 += ht) {
                if (ntiles >= c->max_tiles) return HUFF_ERR_INVALID_ARG;
                c->h_tiles[ntiles++] = HistTile{rec - k, 0, s0, std::min<uint64_t>(r.n, s0 + ht)};
            }
            uint32_t *hist = c->d_hist + hist_words;
            hist_words += (r.nbins + 3) & ~3u;
            uint32_t *st = c->d_status + rec;
            const uintptr_t mis = (16 - ((uintptr_t)r.d_sym & 15)) & 15;
            c->h_hf[rec] = HistField{static_cast<const uint8_t *>(r.d_sym), hist, st, r.nbins,
                                     (uint32_t)(mis / (uintptr_t)r.dtype)};
            c->h_cb[rec] = CbArgs{hist, r.nbins, j.d_book, nullptr, st};
            EncField f{};
            f.sym = static_cast<const uint8_t *>(r.d_sym);
            f.book = j.d_book;
            f.out = j.d_out;
            f.offs = j.d_offs;
            f.total_bits = c->d_total + rec;
            f.status = st;
            f.n = r.n;
            f.cap_words = j.cap_words;
            f.chunk_log2 = s->cfg.chunk_log2;
            f.nchunks = (r.n + (1ull << f.chunk_log2) - 1) >> f.chunk_log2;
            f.nbins = r.nbins;
            f.aligned = ((uintptr_t)r.d_sym & 15) == 0;
            c->h_ef[rec] = f;
            g.enc_tiles += (r.n + sub - 1) / sub;
        }
        g.ntiles = ntiles - g.tile_first;
        groups.push_back(g);
        k = e;
    }
    if (groups.size() > kMaxGroupsPerBatch) return HUFF_ERR_INVALID_ARG;
    cudaStream_t st = c->st;
    if (cudaMemcpyAsync(c->d_tiles, c->h_tiles, sizeof(HistTile) * std::max<uint32_t>(1, ntiles),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(c->d_hf, c->h_hf, sizeof(HistField) * nj, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(c->d_cb, c->h_cb, sizeof(CbArgs) * nj, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(c->d_ef, c->h_ef, sizeof(EncField) * nj, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(c->d_hist, 0, 4 * std::max<uint64_t>(1, hist_words), st) != cudaSuccess ||
        cudaMemsetAsync(c->d_status, 0, 4 * nj, st) != cudaSuccess)
        return HUFF_ERR_CUDA;
    for (size_t gi = 0; gi < groups.size(); gi++) {
        const GroupPlan &g = groups[gi];
        int occ_h = 1, occ_c = 1, occ_e = 1;
        huff_status e = histogram_batch_prepare(g.dtype, g.max_nbins, &occ_h);
        if (e == HUFF_OK) e = codebook_batch_prepare(g.max_nbins, &occ_c);
        if (e == HUFF_OK) e = encode_batch_prepare(g.dtype, g.max_nbins, g.count, &occ_e);
        if (e != HUFF_OK) return e;
        if (g.ntiles) {
            const uint32_t grid_h = (uint32_t)std::min<uint64_t>((uint64_t)s->sms * occ_h, g.ntiles);
            e = histogram_batch_launch(g.dtype, c->d_tiles + g.tile_first, g.ntiles, c->d_hf + g.first, g.max_nbins,
                                       grid_h, st);
            if (e != HUFF_OK) return e;
        }
        uint32_t grid_c = (uint32_t)std::min<uint64_t>((uint64_t)s->sms * occ_c, g.count);
        if (g.max_nbins > 4096) grid_c = std::min<uint32_t>(grid_c, kCbScratchCtas);
        e = codebook_batch_launch(c->d_cb + g.first, g.count, g.max_nbins, grid_c,
                                  g.max_nbins > 4096 ? c->d_cbscr : nullptr, c->cbscr_stride, st);
        if (e != HUFF_OK) return e;
        const EncField &f1 = c->h_ef[g.first];
        if (g.count == 1 && encode_scratch_bytes(f1.n, f1.nbins) <= c->escr_bytes) {
            // a group of one job: the single-field encoder (its segment path
            // where the job's codewords allow it)
            e = encode_launch_ex(f1.sym, f1.n, g.dtype, f1.book, f1.nbins, f1.chunk_log2, -1, 0u, f1.out,
                                 f1.cap_words, f1.offs, f1.total_bits, c->d_escr, f1.status, st, 0u, 0u);
            if (e != HUFF_OK) return e;
            continue;
        }
        e = encode_batch_plan_launch(g.dtype, c->d_ef + g.first, g.count, c->d_conf + gi, -1, 8, st);
        if (e != HUFF_OK) return e;
        if (cudaMemsetAsync(c->d_escr, 0, 64 + 16 * g.enc_tiles, st) != cudaSuccess) return HUFF_ERR_CUDA;
        e = encode_batch_launch(g.dtype, c->d_ef + g.first, g.count, c->d_conf + gi, g.max_nbins, c->d_escr,
                                (uint32_t)(s->sms * occ_e), st);
        if (e != HUFF_OK) return e;
    }
    if (cudaMemcpyAsync(c->h_status, c->d_status, 4 * nj, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(c->h_total, c->d_total, 8 * nj, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HUFF_ERR_CUDA;
    return HUFF_OK;
}

void dispatcher_main(huff_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (!s->stop) admit_locked(s);
        Ctx *c = nullptr;
        for (Ctx &x : s->ctxs)
            if (!x.busy) { c = &x; break; }
        if (c && !s->admitted.empty() && !s->stop) {
            // the batch: admitted jobs in order, up to the job and symbol limits
            std::vector<Job *> jb;
            std::vector<uint64_t> tk;
            uint64_t syms = 0;
            while (!s->admitted.empty() && jb.size() < s->cfg.max_batch) {
                Job &j = s->jobs[s->admitted.front()];
                if (!jb.empty() && syms + j.rq.n > s->cfg.max_batch_symbols) break;
                syms += j.rq.n;
                j.state = JobState::Launched;
                j.t_launch = now_s();
                jb.push_back(&j);
                tk.push_back(s->admitted.front());
                s->admitted.pop_front();
            }
            c->busy = true;
            s->running++;
            s->stats.batches++;
            s->stats.max_batch_jobs = std::max<uint64_t>(s->stats.max_batch_jobs, jb.size());
            s->stats.max_concurrent_batches = std::max(s->stats.max_concurrent_batches, s->running);
            lk.unlock();
            // Job pointers stay valid: a launched job is erased only by its completion.
            huff_status e = launch_batch(s, c, jb, tk);
            if (e == HUFF_OK && cudaLaunchHostFunc(c->st, batch_done, c) != cudaSuccess) e = HUFF_ERR_CUDA;
            if (e != HUFF_OK) cudaStreamSynchronize(c->st);   // nothing of the failed batch may still run
            lk.lock();
            if (e != HUFF_OK) {
                const double t = now_s();
                for (uint64_t tkt : tk) finish_locked(s, tkt, e, 0, t);
                c->tickets.clear();
                c->busy = false;
                s->running--;
                s->cv_done.notify_all();
            }
            continue;
        }
        if (s->stop && s->running == 0) break;
        s->cv.wait(lk);
    }
}

void free_server(huff_server *s) {
    for (Ctx &c : s->ctxs) {
        if (c.st) {
            cudaStreamSynchronize(c.st);
            cudaStreamDestroy(c.st);
        }
        if (c.dmem) cudaFree(c.dmem);
        if (c.hmem) cudaFreeHost(c.hmem);
    }
    if (s->pool_base) cudaFree(s->pool_base);
    delete s;
}

bool request_ok(const huff_server *s, const huff_request *r) {
    if (!r) return false;
    const huff_dtype d = r->dtype;
    if (d != HUFF_U8 && d != HUFF_U16 && d != HUFF_U32) return false;
    if (r->nbins < 1 || r->nbins > HUFF_MAX_BINS_BATCH || (d == HUFF_U8 && r->nbins > 256)) return false;
    if (r->n < 1 || r->n > s->cfg.max_batch_symbols || r->n >= (1ull << 32) || !r->d_sym) return false;
    if (((uintptr_t)r->d_sym % (uintptr_t)d) != 0) return false;
    return true;
}

void fill_result(const Job &j, int m, huff_result *res) {
    res->status = j.status;
    res->chunk_log2 = m;
    res->total_bits = j.total_bits;
    res->d_out = j.d_out;
    res->d_chunk_bit_offset = j.d_offs;
    res->d_codebook = j.d_book;
    res->t_submit = j.t_submit;
    res->t_admit = j.t_admit;
    res->t_launch = j.t_launch;
    res->t_done = j.t_done;
}

}  // namespace

extern "C" {

void huff_serve_default_cfg(huff_serve_cfg *c) {
    if (!c) return;
    c->mem_budget_bytes = 1ull << 30;
    c->max_inflight = 4096;
    c->nstreams = 2;
    c->max_batch = 64;
    c->chunk_log2 = 10;
    c->max_batch_symbols = 1ull << 31;
    c->max_queue = 1u << 20;
    c->reserved = 0;
}

huff_status huff_serve_create(const huff_serve_cfg *cfg, huff_server **out) {
    if (!out) return HUFF_ERR_INVALID_ARG;
    *out = nullptr;
    huff_serve_cfg c;
    huff_serve_default_cfg(&c);
    if (cfg) {
        c = *cfg;
        if (!c.max_inflight) c.max_inflight = 4096;
        if (!c.nstreams) c.nstreams = 2;
        if (!c.max_batch) c.max_batch = 64;
        if (!c.chunk_log2) c.chunk_log2 = 10;
        if (!c.max_batch_symbols) c.max_batch_symbols = 1ull << 31;
        if (!c.max_queue) c.max_queue = 1u << 20;
    }
    if (c.mem_budget_bytes < 4096 || c.nstreams > 16 || c.max_batch > 512 || c.chunk_log2 < 4 ||
        c.chunk_log2 > 30 || c.max_batch_symbols > (1ull << 34))
        return HUFF_ERR_INVALID_ARG;
    huff_server *s = new (std::nothrow) huff_server();
    if (!s) return HUFF_ERR_OOM;
    s->cfg = c;
    cudaGetDevice(&s->device);
    s->sms = sm_count();
    if (cudaMalloc(&s->pool_base, c.mem_budget_bytes) != cudaSuccess) {
        s->pool_base = nullptr;
        free_server(s);
        return HUFF_ERR_OOM;
    }
    s->pool.reset(c.mem_budget_bytes, 256);
    s->stats.pool_capacity = c.mem_budget_bytes;
    // stream contexts: records, histograms, descriptors and scratch for one batch each
    const uint64_t max_tiles = c.max_batch_symbols / 32768 + c.max_batch + 1;
    const uint64_t enc_tiles = c.max_batch_symbols / 2048 + c.max_batch + 1;
    const size_t cbscr_stride = align256(codebook_array_bytes(HUFF_MAX_BINS_BATCH));
    s->ctxs.resize(c.nstreams);
    for (Ctx &x : s->ctxs) {
        x.srv = s;
        x.max_tiles = max_tiles;
        x.cbscr_stride = cbscr_stride;
        size_t off = 0;
        auto take = [&](size_t b) { const size_t at = off; off += align256(b); return at; };
        const size_t o_tiles = take(sizeof(HistTile) * max_tiles), o_hf = take(sizeof(HistField) * c.max_batch),
                     o_cb = take(sizeof(CbArgs) * c.max_batch), o_ef = take(sizeof(EncField) * c.max_batch),
                     o_conf = take(sizeof(EncBatchConf) * kMaxGroupsPerBatch),
                     o_hist = take(4ull * HUFF_MAX_BINS_BATCH * c.max_batch), o_status = take(4ull * c.max_batch),
                     o_total = take(8ull * c.max_batch), o_escr = take(64 + 16 * enc_tiles),
                     o_cbscr = take(cbscr_stride * kCbScratchCtas);
        if (cudaMalloc(&x.dmem, off) != cudaSuccess) {
            x.dmem = nullptr;
            free_server(s);
            return HUFF_ERR_OOM;
        }
        size_t hoff = 0;
        auto htake = [&](size_t b) { const size_t at = hoff; hoff += align256(b); return at; };
        const size_t h_tiles = htake(sizeof(HistTile) * max_tiles), h_hf = htake(sizeof(HistField) * c.max_batch),
                     h_cb = htake(sizeof(CbArgs) * c.max_batch), h_ef = htake(sizeof(EncField) * c.max_batch),
                     h_status = htake(4ull * c.max_batch), h_total = htake(8ull * c.max_batch);
        if (cudaMallocHost(&x.hmem, hoff) != cudaSuccess) {
            x.hmem = nullptr;
            free_server(s);
            return HUFF_ERR_OOM;
        }
        if (cudaStreamCreateWithFlags(&x.st, cudaStreamNonBlocking) != cudaSuccess) {
            x.st = nullptr;
            free_server(s);
            return HUFF_ERR_CUDA;
        }
        x.d_tiles = reinterpret_cast<HistTile *>(x.dmem + o_tiles);
        x.d_hf = reinterpret_cast<HistField *>(x.dmem + o_hf);
        x.d_cb = reinterpret_cast<CbArgs *>(x.dmem + o_cb);
        x.d_ef = reinterpret_cast<EncField *>(x.dmem + o_ef);
        x.d_conf = reinterpret_cast<EncBatchConf *>(x.dmem + o_conf);
        x.d_hist = reinterpret_cast<uint32_t *>(x.dmem + o_hist);
        x.d_status = reinterpret_cast<uint32_t *>(x.dmem + o_status);
        x.d_total = reinterpret_cast<uint64_t *>(x.dmem + o_total);
        x.d_escr = x.dmem + o_escr;
        x.escr_bytes = align256(64 + 16 * enc_tiles);
        x.d_cbscr = x.dmem + o_cbscr;
        x.h_tiles = reinterpret_cast<HistTile *>(x.hmem + h_tiles);
        x.h_hf = reinterpret_cast<HistField *>(x.hmem + h_hf);
        x.h_cb = reinterpret_cast<CbArgs *>(x.hmem + h_cb);
        x.h_ef = reinterpret_cast<EncField *>(x.hmem + h_ef);
        x.h_status = reinterpret_cast<uint32_t *>(x.hmem + h_status);
        x.h_total = reinterpret_cast<uint64_t *>(x.hmem + h_total);
    }
    try {
        s->dispatcher = std::thread(dispatcher_main, s);
    } catch (...) {
        free_server(s);
        return HUFF_ERR_OOM;
    }
    *out = s;
    return HUFF_OK;
}

huff_status huff_serve_submit(huff_server *s, const huff_request *r, uint64_t *ticket) {
    if (!s || !ticket || !request_ok(s, r)) return HUFF_ERR_INVALID_ARG;
    const uint64_t bytes = job_bytes(s, *r);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (!s->pool.fits_ever(bytes)) return HUFF_ERR_OOM;
        if (s->stop || s->queue.size() >= s->cfg.max_queue) return HUFF_ERR_BUSY;
        const uint64_t t = s->next_ticket++;
        Job &j = s->jobs[t];
        j.rq = *r;
        j.t_submit = now_s();
        s->queue.push_back(t);
        s->stats.submitted++;
        *ticket = t;
    }
    s->cv.notify_all();
    return HUFF_OK;
}

huff_status huff_serve_poll(huff_server *s, uint64_t ticket, huff_result *res) {
    if (!s || !res) return HUFF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end() || it->second.release_when_done) return HUFF_ERR_NOT_FOUND;
    if (it->second.state != JobState::Done) return HUFF_ERR_BUSY;
    fill_result(it->second, s->cfg.chunk_log2, res);
    return HUFF_OK;
}

huff_status huff_serve_wait(huff_server *s, uint64_t ticket, huff_result *res) {
    if (!s || !res) return HUFF_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end() || it->second.release_when_done) return HUFF_ERR_NOT_FOUND;
        if (it->second.state == JobState::Done) {
            fill_result(it->second, s->cfg.chunk_log2, res);
            return HUFF_OK;
        }
        s->cv_done.wait(lk);
    }
}

huff_status huff_serve_release(huff_server *s, uint64_t ticket) {
    if (!s) return HUFF_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->jobs.find(ticket);
        if (it == s->jobs.end() || it->second.release_when_done) return HUFF_ERR_NOT_FOUND;
        Job &j = it->second;
        if (j.state != JobState::Done) {
            j.release_when_done = true;
            return HUFF_OK;
        }
        free_job_memory(s, j);
        if (j.holds_slot) s->inflight--;
        s->jobs.erase(it);
        s->stats.pool_used = s->pool.used();
    }
    s->cv.notify_all();
    return HUFF_OK;
}

huff_status huff_serve_get_stats(huff_server *s, huff_serve_stats *st) {
    if (!s || !st) return HUFF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    *st = s->stats;
    st->pool_used = s->pool.used();
    st->pool_peak = s->pool.peak();
    st->pool_capacity = s->pool.capacity();
    return HUFF_OK;
}

huff_status huff_serve_destroy(huff_server *s) {
    if (!s) return HUFF_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        const double t = now_s();
        // jobs not on the device are cancelled
        for (uint64_t tk : s->queue) finish_locked(s, tk, HUFF_ERR_CANCELLED, 0, t);
        for (uint64_t tk : s->admitted) finish_locked(s, tk, HUFF_ERR_CANCELLED, 0, t);
        s->queue.clear();
        s->admitted.clear();
    }
    s->cv.notify_all();
    s->cv_done.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    free_server(s);
    return HUFF_OK;
}

}  // extern "C"
