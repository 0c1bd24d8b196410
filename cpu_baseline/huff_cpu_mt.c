/*
 * Multithreaded CPU Huffman encoder: the CPU comparison of Sec. VI (Table V:
 * multi-thread codebook construction on arrays rather than trees and
 * priority queues; Table VI: multi-thread histogram and encoder, scaled over
 * cores).  The paper used OpenMP; this is plain C with POSIX threads, one
 * team of T threads per call (thread 0 is the caller), phases separated by a
 * barrier.
 *
 * It is a reported baseline, not the product and not the oracle: it shares
 * no code with either.  Its results must equal the oracle's bit for bit, so
 * it follows the same definitions:
 *   - lengths: Huffman's construction with two queues over the used symbols
 *     sorted by (count, id); on equal weight the leaf is taken first;
 *   - codes: canonical, longest length first from 0 (first[max] = 0,
 *     first[l] = ceil((first[l+1] + count[l+1]) / 2)), ascending id within
 *     one length;
 *   - stream: codewords in input order, most significant bit first, packed
 *     into 32-bit words from bit 31 of word 0; the tail of the last word is
 *     zero; chunk_bit_offset[c] is the stream position of symbol c * 2^M and
 *     the final entry is the total.
 *
 * Return codes: 0 ok, -1 invalid argument, -2 symbol >= nbins, -3 symbol
 * without a codeword, -4 output capacity too small, -5 counts sum >= 2^32,
 * -7 thread creation failed.
 */
#define _GNU_SOURCE
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MT_MAX_THREADS 256
#define MT_MAX_LEN 64

/* ------------------------------------------------------------------ team */

typedef struct team team_t;
typedef void (*body_fn)(team_t *tm, int t, void *ctx);

struct team {
    int T;
    pthread_barrier_t bar;
    body_fn fn;
    void *ctx;
    pthread_mutex_t mu;
    pthread_cond_t cv;
    int state;               /* 0: threads being created, 1: go, -1: abandon */
};

typedef struct { team_t *tm; int t; } arg_t;

static void *team_entry(void *p)
{
    arg_t *a = (arg_t *)p;
    team_t *tm = a->tm;
    pthread_mutex_lock(&tm->mu);
    while (tm->state == 0) pthread_cond_wait(&tm->cv, &tm->mu);
    const int go = tm->state == 1;
    pthread_mutex_unlock(&tm->mu);
    if (go) tm->fn(tm, a->t, tm->ctx);
    return NULL;
}

static void team_sync(team_t *tm)
{
    if (tm->T > 1) pthread_barrier_wait(&tm->bar);
}

/* Runs fn(t) on threads t = 0..T-1 (0 on the caller) and joins them.  No
 * thread starts fn before all T exist, so a failed thread creation abandons
 * the call (-7) instead of leaving a barrier that never completes. */
static int team_run(int T, body_fn fn, void *ctx)
{
    team_t tm;
    tm.T = T;
    tm.fn = fn;
    tm.ctx = ctx;
    if (T == 1) { fn(&tm, 0, ctx); return 0; }
    if (pthread_barrier_init(&tm.bar, NULL, (unsigned)T) != 0) return -7;
    pthread_mutex_init(&tm.mu, NULL);
    pthread_cond_init(&tm.cv, NULL);
    tm.state = 0;
    pthread_t th[MT_MAX_THREADS];
    arg_t args[MT_MAX_THREADS];
    int started = 0;
    for (int t = 1; t < T; t++) {
        args[t].tm = &tm;
        args[t].t = t;
        if (pthread_create(&th[t], NULL, team_entry, &args[t]) != 0) break;
        started++;
    }
    const int ok = started == T - 1;
    pthread_mutex_lock(&tm.mu);
    tm.state = ok ? 1 : -1;
    pthread_cond_broadcast(&tm.cv);
    pthread_mutex_unlock(&tm.mu);
    if (ok) fn(&tm, 0, ctx);
    for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
    pthread_barrier_destroy(&tm.bar);
    pthread_cond_destroy(&tm.cv);
    pthread_mutex_destroy(&tm.mu);
    return ok ? 0 : -7;
}

static void split(uint64_t n, int T, int t, uint64_t *lo, uint64_t *hi)
{
    *lo = n * (uint64_t)t / (uint64_t)T;
    *hi = n * (uint64_t)(t + 1) / (uint64_t)T;
}

/* -------------------------------------------------------------- histogram */

typedef struct {
    const void *sym;
    uint64_t n;
    int width;
    uint32_t nbins;
    uint32_t *hist;
    uint32_t *priv;          /* T private histograms of nbins counts */
    int err[MT_MAX_THREADS];
} hist_ctx;

/* Phase 1: each thread counts a contiguous block into its own histogram,
 * spread over four sub-histograms (consecutive symbols go to different ones,
 * so runs of equal symbols do not serialise on one counter).
 * Phase 2: each thread sums a range of bins over all sub-histograms. */
#define HIST_LOOP(T)                                                                 \
    do {                                                                             \
        const T *s = (const T *)c->sym;                                              \
        uint64_t i = lo;                                                             \
        for (; i + 4 <= hi; i += 4) {                                                \
            const uint32_t v0 = s[i], v1 = s[i + 1], v2 = s[i + 2], v3 = s[i + 3];   \
            if ((v0 | v1 | v2 | v3) < nb || (v0 < nb && v1 < nb && v2 < nb && v3 < nb)) { \
                h0[v0]++; h1[v1]++; h2[v2]++; h3[v3]++;                              \
            } else {                                                                 \
                bad = 1;                                                             \
            }                                                                        \
        }                                                                            \
        for (; i < hi; i++) {                                                        \
            const uint32_t v = s[i];                                                 \
            if (v < nb) h0[v]++; else bad = 1;                                       \
        }                                                                            \
    } while (0)

static void hist_body(team_t *tm, int t, void *p)
{
    hist_ctx *c = (hist_ctx *)p;
    const uint32_t nb = c->nbins;
    uint32_t *h0 = c->priv + (uint64_t)t * 4 * nb, *h1 = h0 + nb, *h2 = h1 + nb, *h3 = h2 + nb;
    memset(h0, 0, sizeof(uint32_t) * 4 * nb);
    uint64_t lo, hi;
    split(c->n, tm->T, t, &lo, &hi);
    int bad = 0;
    if (c->width == 2) HIST_LOOP(uint16_t);
    else if (c->width == 1) HIST_LOOP(uint8_t);
    else HIST_LOOP(uint32_t);
    c->err[t] = bad ? -2 : 0;
    team_sync(tm);
    uint64_t b0, b1;
    split(nb, tm->T, t, &b0, &b1);
    for (uint64_t k = b0; k < b1; k++) {
        uint32_t sum = 0;
        for (int u = 0; u < 4 * tm->T; u++) sum += c->priv[(uint64_t)u * nb + k];
        c->hist[k] = sum;
    }
}
#undef HIST_LOOP

int mt_histogram(const void *sym, uint64_t n, int width, uint32_t nbins, uint32_t *hist, int threads)
{
    if (nbins == 0 || (width != 1 && width != 2 && width != 4) || threads < 1 || threads > MT_MAX_THREADS ||
        (n && !sym) || !hist)
        return -1;
    if (n < (uint64_t)threads * 4096) threads = (int)(n / 4096) + 1;
    hist_ctx c;
    c.sym = sym; c.n = n; c.width = width; c.nbins = nbins; c.hist = hist;
    c.priv = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nbins * 4 * threads);
    if (!c.priv) return -1;
    int rc = team_run(threads, hist_body, &c);
    if (!rc)
        for (int t = 0; t < threads; t++) if (c.err[t]) rc = c.err[t];
    free(c.priv);
    return rc;
}

/* --------------------------------------------------------------- codebook */

typedef struct {
    const uint32_t *hist;
    uint32_t nbins;
    uint8_t *len;
    uint64_t *code;
    /* used symbols, compacted in id order then sorted by count (stable) */
    uint32_t m;
    uint32_t *ids, *ids2;
    uint32_t *cnt_off;       /* per thread: used symbols in its bin range, then its offset */
    uint32_t *radix;         /* per thread: 256 digit counts */
    uint64_t *lcount;        /* per thread: symbols of each length in its bin range */
    uint64_t first[MT_MAX_LEN + 2];
    uint64_t count[MT_MAX_LEN + 2];
    int maxl;
    int err;
} cb_ctx;

/* Stable LSD radix sort of ids by hist[id], 8 bits a pass; each thread owns a
 * contiguous block of the array, so equal counts keep their id order. */
static void radix_pass(team_t *tm, int t, cb_ctx *c, int shift, uint32_t *src, uint32_t *dst)
{
    uint64_t lo, hi;
    split(c->m, tm->T, t, &lo, &hi);
    uint32_t *r = c->radix + (uint64_t)t * 256;
    memset(r, 0, 256 * sizeof(uint32_t));
    for (uint64_t i = lo; i < hi; i++) r[(c->hist[src[i]] >> shift) & 255]++;
    team_sync(tm);
    /* offsets: digit-major, thread-minor */
    uint32_t off[256];
    uint64_t base = 0;
    for (int d = 0; d < 256; d++) {
        for (int u = 0; u < tm->T; u++) {
            if (u == t) off[d] = (uint32_t)base;
            base += c->radix[(uint64_t)u * 256 + d];
        }
    }
    for (uint64_t i = lo; i < hi; i++) dst[off[(c->hist[src[i]] >> shift) & 255]++] = src[i];
    team_sync(tm);
}

static void cb_body(team_t *tm, int t, void *p)
{
    cb_ctx *c = (cb_ctx *)p;
    const int T = tm->T;
    uint64_t b0, b1;
    split(c->nbins, T, t, &b0, &b1);

    /* 1. compact the used symbols in id order */
    uint32_t used = 0;
    for (uint64_t k = b0; k < b1; k++) used += c->hist[k] > 0;
    c->cnt_off[t] = used;
    team_sync(tm);
    if (t == 0) {
        uint32_t s = 0;
        for (int u = 0; u < T; u++) { uint32_t x = c->cnt_off[u]; c->cnt_off[u] = s; s += x; }
        c->m = s;
    }
    team_sync(tm);
    uint32_t w = c->cnt_off[t];
    for (uint64_t k = b0; k < b1; k++)
        if (c->hist[k]) c->ids[w++] = (uint32_t)k;
    for (uint64_t k = b0; k < b1; k++) c->len[k] = 0;
    team_sync(tm);
    if (c->m <= 1) {
        if (t == 0) {
            if (c->m == 1) c->len[c->ids[0]] = 1;
            c->maxl = (int)c->m;
        }
        team_sync(tm);
    } else {
        /* 2. sort by count (stable: ties stay in id order) */
        uint32_t maxc = 0;
        for (uint32_t i = 0; i < c->m; i++) if (c->hist[c->ids[i]] > maxc) maxc = c->hist[c->ids[i]];
        uint32_t *src = c->ids, *dst = c->ids2;
        for (int shift = 0; shift < 32 && (shift == 0 || (maxc >> shift)); shift += 8) {
            radix_pass(tm, t, c, shift, src, dst);
            uint32_t *x = src; src = dst; dst = x;
        }
        /* 3. lengths: the two-queue merge is one linear pass (thread 0) */
        if (t == 0) {
            const uint32_t m = c->m;
            uint64_t *iw = (uint64_t *)malloc(sizeof(uint64_t) * (m - 1));
            uint32_t *par = (uint32_t *)malloc(sizeof(uint32_t) * (2 * m - 1));
            uint32_t *dep = (uint32_t *)malloc(sizeof(uint32_t) * (2 * m - 1));
            if (!iw || !par || !dep) {
                c->err = -1;
            } else {
                uint32_t a = 0, b = 0, e = 0;   /* next leaf, next joined node, joined nodes made */
                for (uint32_t j = 0; j + 1 < m; j++) {
                    uint64_t sum = 0;
                    for (int q = 0; q < 2; q++) {
                        int leaf = a < m && (b >= e || (uint64_t)c->hist[src[a]] <= iw[b]);
                        uint32_t node;
                        if (leaf) { node = a; sum += c->hist[src[a]]; a++; }
                        else { node = m + b; sum += iw[b]; b++; }
                        par[node] = m + e;
                    }
                    iw[e++] = sum;
                }
                dep[2 * m - 2] = 0;
                for (int64_t v = (int64_t)(2 * m) - 3; v >= 0; v--) dep[v] = dep[par[v]] + 1;
                int maxl = 0;
                for (uint32_t v = 0; v < m; v++) {
                    if (dep[v] > MT_MAX_LEN) c->err = -1;
                    else c->len[src[v]] = (uint8_t)dep[v];
                    if ((int)dep[v] > maxl) maxl = (int)dep[v];
                }
                c->maxl = maxl;
            }
            free(iw); free(par); free(dep);
        }
        team_sync(tm);
    }
    if (c->err || c->maxl == 0) return;

    /* 4. canonical codes: per-thread counts of each length over its bins */
    uint64_t *lc = c->lcount + (uint64_t)t * (MT_MAX_LEN + 1);
    memset(lc, 0, sizeof(uint64_t) * (MT_MAX_LEN + 1));
    for (uint64_t k = b0; k < b1; k++) if (c->len[k]) lc[c->len[k]]++;
    team_sync(tm);
    if (t == 0) {
        memset(c->count, 0, sizeof(c->count));
        for (int u = 0; u < T; u++)
            for (int l = 1; l <= MT_MAX_LEN; l++) c->count[l] += c->lcount[(uint64_t)u * (MT_MAX_LEN + 1) + l];
        memset(c->first, 0, sizeof(c->first));
        for (int l = c->maxl - 1; l >= 1; l--) c->first[l] = (c->first[l + 1] + c->count[l + 1] + 1) >> 1;
    }
    team_sync(tm);
    uint64_t next[MT_MAX_LEN + 1];
    for (int l = 1; l <= MT_MAX_LEN; l++) {
        uint64_t before = 0;
        for (int u = 0; u < t; u++) before += c->lcount[(uint64_t)u * (MT_MAX_LEN + 1) + l];
        next[l] = c->first[l] + before;
    }
    for (uint64_t k = b0; k < b1; k++) {
        const int l = c->len[k];
        c->code[k] = l ? next[l]++ : 0;
    }
}

int mt_codebook(const uint32_t *hist, uint32_t nbins, uint8_t *len, uint64_t *code, int threads)
{
    if (!hist || !len || !code || nbins == 0 || threads < 1 || threads > MT_MAX_THREADS) return -1;
    uint64_t total = 0;
    for (uint32_t k = 0; k < nbins; k++) total += hist[k];
    if (total >= (1ull << 32)) return -5;
    if (nbins < (uint32_t)threads * 64) threads = (int)(nbins / 64) + 1;
    cb_ctx c;
    memset(&c, 0, sizeof(c));
    c.hist = hist; c.nbins = nbins; c.len = len; c.code = code;
    c.ids = (uint32_t *)malloc(sizeof(uint32_t) * nbins);
    c.ids2 = (uint32_t *)malloc(sizeof(uint32_t) * nbins);
    c.cnt_off = (uint32_t *)malloc(sizeof(uint32_t) * threads);
    c.radix = (uint32_t *)malloc(sizeof(uint32_t) * 256 * threads);
    c.lcount = (uint64_t *)malloc(sizeof(uint64_t) * (MT_MAX_LEN + 1) * threads);
    int rc = -1;
    if (c.ids && c.ids2 && c.cnt_off && c.radix && c.lcount) {
        rc = team_run(threads, cb_body, &c);
        if (!rc) rc = c.err ? c.err : c.maxl;
    }
    if (rc == 0) for (uint32_t k = 0; k < nbins; k++) code[k] = 0;
    free(c.ids); free(c.ids2); free(c.cnt_off); free(c.radix); free(c.lcount);
    return rc;
}

/* ----------------------------------------------------------------- encode */

typedef struct {
    const void *sym;
    uint64_t n;
    int width;
    const uint64_t *code;
    const uint8_t *len;
    uint32_t nbins;
    int chunk_log2;
    uint64_t nchunks;
    uint32_t max_len;
    uint32_t *out;
    uint64_t cap;
    uint64_t *offs;
    uint32_t *priv[MT_MAX_THREADS];     /* each thread's stream, from bit 0 of its own buffer */
    uint64_t tbits[MT_MAX_THREADS];     /* bits of each thread's chunk range, then its start */
    uint64_t edge_idx[MT_MAX_THREADS][2];
    uint32_t edge_val[MT_MAX_THREADS][2];
    int nedge[MT_MAX_THREADS];
    int err[MT_MAX_THREADS];
    uint64_t total;
} enc_ctx;

/* Packs symbols [i0, i1) (chunk-aligned at i0) into buf from bit 0, most
 * significant bit first; offs[c] receives each chunk's start relative to the
 * buffer.  acc holds the nb (< 32) pending bits left-aligned at bit 63.  A
 * code of at most 32 bits is placed below them, the top 32 bits of acc are
 * stored to buf[w] unconditionally (a partial word is rewritten until it is
 * complete), and w advances by one when 32 bits are done: no branch on the
 * word boundary.  Longer codes (rare) go in two halves.  Returns the bit
 * count, or a negative error. */
#define PACK_FN(NAME, T)                                                                          \
static int64_t NAME(const T *s, uint64_t i0, uint64_t i1, uint64_t chunk, const uint64_t *code,   \
                    const uint8_t *len, uint32_t nbins, uint32_t *buf, uint64_t *offs)            \
{                                                                                                 \
    uint64_t acc = 0, w = 0;                                                                      \
    uint32_t nb = 0;                                                                              \
    buf[0] = 0;                                                                                   \
    for (uint64_t c0 = i0; c0 < i1; c0 += chunk) {                                                \
        *offs++ = 32 * w + nb;                                                                    \
        const uint64_t ce = c0 + chunk < i1 ? c0 + chunk : i1;                                    \
        for (uint64_t i = c0; i < ce; i++) {                                                      \
            const uint32_t v = s[i];                                                              \
            if (v >= nbins) return -2;                                                            \
            uint32_t l = len[v];                                                                  \
            uint64_t cw = code[v];                                                                \
            if (l - 1u >= 32u) {                   /* 0 (no codeword) or longer than 32 bits */   \
                if (l == 0) return -3;                                                            \
                const uint32_t h = l - 32;                                                        \
                acc |= (cw >> 32) << (64 - nb - h);                                               \
                nb += h;                                                                          \
                buf[w] = (uint32_t)(acc >> 32);                                                   \
                if (nb >= 32) { w++; acc <<= 32; nb -= 32; }                                      \
                cw &= 0xFFFFFFFFull;                                                              \
                l = 32;                                                                           \
            }                                                                                     \
            acc |= cw << (64 - nb - l);            /* nb + l <= 63 */                             \
            nb += l;                                                                              \
            buf[w] = (uint32_t)(acc >> 32);                                                       \
            const uint32_t f = nb >> 5;            /* 1 when a word is done */                    \
            w += f;                                                                               \
            acc <<= 32 * f;                                                                       \
            nb -= 32 * f;                                                                         \
        }                                                                                         \
    }                                                                                             \
    buf[w] = (uint32_t)(acc >> 32);                /* zero-padded tail (zero if nb = 0) */         \
    buf[w + 1] = 0;                                                                               \
    return (int64_t)(32 * w + nb);                                                                \
}
PACK_FN(pack_u8, uint8_t)
PACK_FN(pack_u16, uint16_t)
PACK_FN(pack_u32, uint32_t)
#undef PACK_FN

/* Phase 1: each thread packs its chunk range into its own buffer (the input
 * is read once) and records chunk starts relative to it.  Thread 0 scans the
 * range totals.  Phase 2: chunk starts become stream offsets and each buffer
 * is copied to the stream at its start bit, shifted into place; words wholly
 * inside the range are stored directly, and the (at most two) words shared
 * with a neighbour are handed back and OR-ed in by the caller after the join. */
static void enc_body(team_t *tm, int t, void *p)
{
    enc_ctx *c = (enc_ctx *)p;
    uint64_t c0, c1;
    split(c->nchunks, tm->T, t, &c0, &c1);
    const uint64_t chunk = 1ull << c->chunk_log2;
    const uint64_t i0 = c0 * chunk, i1 = c1 * chunk < c->n ? c1 * chunk : c->n;
    uint32_t *buf = c->priv[t];
    int64_t bits = 0;
    if (i1 > i0) {
        switch (c->width) {
            case 1: bits = pack_u8((const uint8_t *)c->sym, i0, i1, chunk, c->code, c->len, c->nbins, buf, c->offs + c0); break;
            case 2: bits = pack_u16((const uint16_t *)c->sym, i0, i1, chunk, c->code, c->len, c->nbins, buf, c->offs + c0); break;
            default: bits = pack_u32((const uint32_t *)c->sym, i0, i1, chunk, c->code, c->len, c->nbins, buf, c->offs + c0); break;
        }
    }
    c->err[t] = bits < 0 ? (int)bits : 0;
    c->tbits[t] = bits < 0 ? 0 : (uint64_t)bits;
    team_sync(tm);
    if (t == 0) {
        uint64_t sum = 0;
        int any = 0;
        for (int u = 0; u < tm->T; u++) { uint64_t x = c->tbits[u]; c->tbits[u] = sum; sum += x; any |= c->err[u]; }
        c->total = sum;
        if (!any && (sum + 31) / 32 > c->cap) c->err[0] = -4;
    }
    team_sync(tm);
    for (int u = 0; u < tm->T; u++) if (c->err[u]) return;

    const uint64_t base = c->tbits[t];
    const uint64_t B = (uint64_t)bits;
    for (uint64_t ch = c0; ch < c1; ch++) c->offs[ch] += base;
    c->nedge[t] = 0;
    if (B == 0) return;
    const uint32_t sh = (uint32_t)(base & 31);
    const uint64_t w0 = base >> 5, w1 = (base + B - 1) >> 5;     /* output words touched */
    const int head_shared = sh != 0, tail_shared = ((base + B) & 31) != 0;
    for (uint64_t j = w0; j <= w1; j++) {
        const uint64_t k = j - w0;
        const uint32_t cur = buf[k];
        const uint32_t v = sh ? ((k ? buf[k - 1] << (32 - sh) : 0u) | (cur >> sh)) : cur;
        if ((j == w0 && head_shared) || (j == w1 && tail_shared)) {
            c->edge_idx[t][c->nedge[t]] = j;
            c->edge_val[t][c->nedge[t]++] = v;
        } else {
            c->out[j] = v;
        }
    }
}

int mt_encode(const void *sym, uint64_t n, int width, const uint64_t *code, const uint8_t *len, uint32_t nbins,
              int chunk_log2, uint32_t *out, uint64_t out_cap_words, uint64_t *chunk_bit_offset,
              uint64_t *total_bits, int threads)
{
    if (chunk_log2 < 0 || chunk_log2 > 40 || (width != 1 && width != 2 && width != 4) || threads < 1 ||
        threads > MT_MAX_THREADS || !code || !len || !chunk_bit_offset || !total_bits || (n && (!sym || !out)))
        return -1;
    enc_ctx *c = (enc_ctx *)calloc(1, sizeof(enc_ctx));
    if (!c) return -1;
    c->sym = sym; c->n = n; c->width = width; c->code = code; c->len = len; c->nbins = nbins;
    c->chunk_log2 = chunk_log2; c->out = out; c->cap = out_cap_words; c->offs = chunk_bit_offset;
    c->nchunks = (n + (1ull << chunk_log2) - 1) >> chunk_log2;
    uint32_t maxl = 0;
    for (uint32_t k = 0; k < nbins; k++) if (len[k] > maxl) maxl = len[k];
    c->max_len = maxl;
    if (c->nchunks < (uint64_t)threads) threads = c->nchunks ? (int)c->nchunks : 1;
    int rc = 0;
    for (int t = 0; t < threads && !rc; t++) {
        uint64_t a, b;
        split(c->nchunks, threads, t, &a, &b);
        uint64_t lo = a << chunk_log2, hi = (b << chunk_log2) < n ? (b << chunk_log2) : n;
        uint64_t syms = hi > lo ? hi - lo : 0;
        /* worst case: every symbol at the longest length; pages are touched only as written */
        c->priv[t] = (uint32_t *)malloc(sizeof(uint32_t) * ((syms * (maxl ? maxl : 1) + 31) / 32 + 2));
        if (!c->priv[t]) rc = -1;
    }
    if (!rc) rc = team_run(threads, enc_body, c);
    for (int t = 0; t < threads && !rc; t++) if (c->err[t]) rc = c->err[t];
    if (!rc) {
        for (int t = 0; t < threads; t++)
            for (int e = 0; e < c->nedge[t]; e++) out[c->edge_idx[t][e]] = 0;
        for (int t = 0; t < threads; t++)
            for (int e = 0; e < c->nedge[t]; e++) out[c->edge_idx[t][e]] |= c->edge_val[t][e];
        chunk_bit_offset[c->nchunks] = c->total;
        *total_bits = c->total;
    }
    for (int t = 0; t < threads; t++) free(c->priv[t]);
    free(c);
    return rc;
}
