/*
 * CPU oracle for the Huffman encoding pipeline of "Revisiting Huffman Coding:
 * Toward Extreme Performance on Modern GPU Architectures" (Tian et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or helper with the CUDA library; it is a plain, serial,
 * obviously-correct restatement of what the paper's pipeline computes:
 *
 *   oracle_histogram          Sec. IV-A     counts of each symbol
 *   oracle_lengths_two_queue  Sec. IV-B1    optimal code lengths (Huffman's
 *                                           construction, van Leeuwen's
 *                                           two-queue form, leaf first on ties)
 *   oracle_lengths_heap       Sec. IV-B1    the same rule with a binary heap
 *                                           (independent second formulation)
 *   oracle_canonical          Sec. IV-B2    canonical codewords from lengths
 *                                           plus First/Entry decode metadata
 *   oracle_encode             Sec. IV-C     codeword concatenation (the Merge
 *                                           operator's order: a_{2k+1} right
 *                                           after a_{2k}) into one dense
 *                                           MSB-first bitstream, chunk offsets
 *   oracle_encode_format      Sec. IV-C,    the same concatenation written as
 *                             Sec. VI       typed units of W = 8, 16 or 32
 *                                           bits, dense or with every chunk
 *                                           starting at a unit boundary (the
 *                                           un-gathered chunks)
 *   oracle_decode             Sec. IV-B2    treeless canonical decoding with
 *                                           First and Entry
 *
 * Readings taken where the paper is silent:
 *  - symbols with zero count get no codeword (length 0);
 *  - a single used symbol gets length 1 and codeword 0;
 *  - ties in the tree construction: leaves are ordered by (count, id); when a
 *    leaf and an internal node have equal weight the leaf is taken first;
 *    internal nodes leave their queue in creation order;
 *  - canonical orientation as Sec. IV-B2 asks (a short codeword is numerically
 *    larger than the same-length prefix of any longer one), codewords of one
 *    length in ascending symbol id;
 *  - the bitstream is an array of 32-bit words, bit 31 of word 0 first;
 *  - a stream of W-bit typed units holds the same bits, bit W-1 of unit 0
 *    first; in the chunk-aligned form a chunk's last unit is padded with zero
 *    bits and its offset counts units, and the stream's length counts the
 *    padding.
 *
 * Error returns (negative): -1 bad argument, -2 symbol >= nbins, -3 symbol
 * without codeword, -4 output capacity too small, -5 histogram sum >= 2^32,
 * -6 undecodable stream.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_LEN 64

static uint32_t load_sym(const void *sym, uint64_t i, int width)
{
    if (width == 1) return ((const uint8_t *)sym)[i];
    if (width == 2) return ((const uint16_t *)sym)[i];
    return ((const uint32_t *)sym)[i];
}

/* ---------------------------------------------------------------- histogram */

int oracle_histogram(const void *sym, uint64_t n, int width, uint32_t nbins, uint32_t *hist)
{
    if (nbins == 0 || (width != 1 && width != 2 && width != 4)) return -1;
    memset(hist, 0, sizeof(uint32_t) * nbins);
    for (uint64_t i = 0; i < n; i++) {
        uint32_t s = load_sym(sym, i, width);
        if (s >= nbins) return -2;
        hist[s] += 1;
    }
    return 0;
}

/* ------------------------------------------------------ lengths: two queues */

typedef struct { uint64_t w; uint32_t id; } leaf_t;

static int leaf_cmp(const void *a, const void *b)
{
    const leaf_t *x = (const leaf_t *)a, *y = (const leaf_t *)b;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

static int check_sum(const uint32_t *hist, uint32_t nbins)
{
    uint64_t total = 0;
    for (uint32_t k = 0; k < nbins; k++) total += hist[k];
    return total >= (1ull << 32) ? -5 : 0;
}

/*
 * Huffman's construction: repeatedly join the two lightest nodes.  Leaves wait
 * in a queue sorted by (count, id); joined nodes are appended to a second
 * queue, which stays sorted by weight because each join is at least as heavy
 * as the one before.  Each step takes the lighter queue head, the leaf on
 * equal weight.  A leaf's length is its depth in the finished tree.
 * Returns the longest length (0 if no symbol is used) or a negative error.
 */
int oracle_lengths_two_queue(const uint32_t *hist, uint32_t nbins, uint8_t *len)
{
    if (nbins == 0) return -1;
    int rc = check_sum(hist, nbins);
    if (rc) return rc;
    memset(len, 0, nbins);
    uint32_t m = 0;
    for (uint32_t k = 0; k < nbins; k++) m += hist[k] > 0;
    if (m == 0) return 0;
    leaf_t *leaf = (leaf_t *)malloc(sizeof(leaf_t) * m);
    uint32_t j = 0;
    for (uint32_t k = 0; k < nbins; k++)
        if (hist[k]) { leaf[j].w = hist[k]; leaf[j].id = k; j++; }
    if (m == 1) { len[leaf[0].id] = 1; free(leaf); return 1; }
    qsort(leaf, m, sizeof(leaf_t), leaf_cmp);

    /* node ids: leaves 0..m-1 (sorted order), joined nodes m..2m-2 */
    uint64_t *iw = (uint64_t *)malloc(sizeof(uint64_t) * (m - 1));
    uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * (2 * m - 1));
    uint32_t lh = 0, ih = 0, it = 0;
    for (uint32_t step = 0; step < m - 1; step++) {
        uint32_t pick[2];
        uint64_t wsum = 0;
        for (int p = 0; p < 2; p++) {
            int take_leaf;
            if (lh >= m) take_leaf = 0;
            else if (ih >= it) take_leaf = 1;
            else take_leaf = leaf[lh].w <= iw[ih];          /* leaf first on ties */
            if (take_leaf) { pick[p] = lh; wsum += leaf[lh].w; lh++; }
            else { pick[p] = m + ih; wsum += iw[ih]; ih++; }
        }
        iw[it] = wsum;
        parent[pick[0]] = m + it;
        parent[pick[1]] = m + it;
        it++;
    }
    /* depth: the root is the last joined node; parents are created after children */
    uint32_t *depth = (uint32_t *)malloc(sizeof(uint32_t) * (2 * m - 1));
    depth[2 * m - 2] = 0;
    for (int64_t v = (int64_t)(2 * m - 3); v >= 0; v--) depth[v] = depth[parent[v]] + 1;
    uint32_t maxl = 0;
    int bad = 0;
    for (uint32_t v = 0; v < m; v++) {
        if (depth[v] > ORACLE_MAX_LEN) bad = 1;
        len[leaf[v].id] = (uint8_t)depth[v];
        if (depth[v] > maxl) maxl = depth[v];
    }
    free(depth); free(parent); free(iw); free(leaf);
    return bad ? -1 : (int)maxl;
}

/* ------------------------------------------------------ lengths: binary heap */

typedef struct { uint64_t w; uint32_t kind; uint32_t seq; uint32_t node; } hent_t;

static int hless(const hent_t *a, const hent_t *b)
{
    if (a->w != b->w) return a->w < b->w;
    if (a->kind != b->kind) return a->kind < b->kind;   /* leaf (0) before joined (1) */
    return a->seq < b->seq;                             /* leaf: symbol id; joined: creation order */
}

static void hpush(hent_t *h, uint32_t *n, hent_t e)
{
    uint32_t i = (*n)++;
    h[i] = e;
    while (i > 0) {
        uint32_t p = (i - 1) / 2;
        if (!hless(&h[i], &h[p])) break;
        hent_t t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static hent_t hpop(hent_t *h, uint32_t *n)
{
    hent_t top = h[0];
    h[0] = h[--(*n)];
    uint32_t i = 0;
    for (;;) {
        uint32_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *n && hless(&h[l], &h[s])) s = l;
        if (r < *n && hless(&h[r], &h[s])) s = r;
        if (s == i) break;
        hent_t t = h[i]; h[i] = h[s]; h[s] = t;
        i = s;
    }
    return top;
}

/*
 * The same selection rule driven by one priority queue keyed on
 * (weight, leaf-before-joined, id or creation order); lengths come from an
 * explicit walk down the finished tree rather than from parent links.
 */
int oracle_lengths_heap(const uint32_t *hist, uint32_t nbins, uint8_t *len)
{
    if (nbins == 0) return -1;
    int rc = check_sum(hist, nbins);
    if (rc) return rc;
    memset(len, 0, nbins);
    uint32_t m = 0;
    for (uint32_t k = 0; k < nbins; k++) m += hist[k] > 0;
    if (m == 0) return 0;
    if (m == 1) {
        for (uint32_t k = 0; k < nbins; k++) if (hist[k]) len[k] = 1;
        return 1;
    }
    /* tree storage: node < nbins is symbol `node`; node >= nbins is joined node (node - nbins) */
    uint32_t *left = (uint32_t *)malloc(sizeof(uint32_t) * (m - 1));
    uint32_t *right = (uint32_t *)malloc(sizeof(uint32_t) * (m - 1));
    hent_t *heap = (hent_t *)malloc(sizeof(hent_t) * m);
    uint32_t hn = 0;
    for (uint32_t k = 0; k < nbins; k++)
        if (hist[k]) { hent_t e = { hist[k], 0, k, k }; hpush(heap, &hn, e); }
    uint32_t made = 0;
    while (hn > 1) {
        hent_t a = hpop(heap, &hn), b = hpop(heap, &hn);
        left[made] = a.node; right[made] = b.node;
        hent_t e = { a.w + b.w, 1, made, nbins + made };
        made++;
        hpush(heap, &hn, e);
    }
    /* iterative depth-first walk from the root */
    uint32_t *stack = (uint32_t *)malloc(sizeof(uint32_t) * 2 * m);
    uint32_t *sdep = (uint32_t *)malloc(sizeof(uint32_t) * 2 * m);
    uint32_t sp = 0, maxl = 0;
    int bad = 0;
    stack[sp] = heap[0].node; sdep[sp] = 0; sp++;
    while (sp) {
        sp--;
        uint32_t v = stack[sp], d = sdep[sp];
        if (v < nbins) {
            if (d > ORACLE_MAX_LEN) bad = 1;
            len[v] = (uint8_t)d;
            if (d > maxl) maxl = d;
        } else {
            uint32_t j = v - nbins;
            stack[sp] = left[j]; sdep[sp] = d + 1; sp++;
            stack[sp] = right[j]; sdep[sp] = d + 1; sp++;
        }
    }
    free(sdep); free(stack); free(heap); free(right); free(left);
    return bad ? -1 : (int)maxl;
}

/* ---------------------------------------------------------------- canonical */

/*
 * Canonical codewords from code lengths, in the orientation Sec. IV-B2 needs
 * for treeless decoding: the longest codewords start at 0, and the first
 * codeword of length l is first[l] = ceil((first[l+1] + count[l+1]) / 2), so
 * that every l-bit prefix of a longer codeword is smaller than first[l].
 * Within one length, symbols get first[l], first[l]+1, ... in ascending id.
 * entry[l] = number of used symbols shorter than l; sorted_syms lists the used
 * symbols by (length, id).  Arrays first/entry/count have 65 slots (index =
 * length).  Returns the longest length, or a negative error.
 */
int oracle_canonical(const uint8_t *len, uint32_t nbins, uint64_t *code, uint64_t *first,
                     uint32_t *entry, uint32_t *count, uint32_t *sorted_syms, uint32_t *nused)
{
    if (nbins == 0) return -1;
    memset(first, 0, sizeof(uint64_t) * (ORACLE_MAX_LEN + 1));
    memset(entry, 0, sizeof(uint32_t) * (ORACLE_MAX_LEN + 1));
    memset(count, 0, sizeof(uint32_t) * (ORACLE_MAX_LEN + 1));
    uint32_t maxl = 0, used = 0;
    for (uint32_t k = 0; k < nbins; k++) {
        if (len[k] > ORACLE_MAX_LEN) return -1;
        if (len[k]) { count[len[k]]++; used++; if (len[k] > maxl) maxl = len[k]; }
    }
    *nused = used;
    for (uint32_t k = 0; k < nbins; k++) code[k] = 0;
    if (maxl == 0) return 0;
    first[maxl] = 0;
    for (int l = (int)maxl - 1; l >= 1; l--)
        first[l] = (first[l + 1] + count[l + 1] + 1) >> 1;
    entry[1] = 0;
    for (uint32_t l = 1; l < ORACLE_MAX_LEN; l++) entry[l + 1] = entry[l] + count[l];
    uint32_t next[ORACLE_MAX_LEN + 1];
    memset(next, 0, sizeof(next));
    for (uint32_t k = 0; k < nbins; k++) {
        uint32_t l = len[k];
        if (!l) continue;
        code[k] = first[l] + next[l];
        sorted_syms[entry[l] + next[l]] = k;
        next[l]++;
    }
    return (int)maxl;
}

/* ------------------------------------------------------------------- encode */

/*
 * Serial concatenation of codewords in input order, most significant bit of
 * each codeword first, into 32-bit words (bit 31 of word 0 is stream bit 0;
 * the unused tail of the last word is zero).  chunk_bit_offset[c] is the
 * stream position of symbol c * 2^chunk_log2; the final entry is total_bits.
 */
int oracle_encode(const void *sym, uint64_t n, int width, const uint64_t *code, const uint8_t *len,
                  uint32_t nbins, int chunk_log2, uint32_t *out, uint64_t out_cap_words,
                  uint64_t *chunk_bit_offset, uint64_t *total_bits)
{
    if (chunk_log2 < 0 || chunk_log2 > 40) return -1;
    uint64_t chunk = 1ull << chunk_log2;
    uint64_t p = 0;
    uint64_t c = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (i % chunk == 0) chunk_bit_offset[c++] = p;
        uint32_t s = load_sym(sym, i, width);
        if (s >= nbins) return -2;
        uint32_t l = len[s];
        if (l == 0) return -3;
        for (int b = (int)l - 1; b >= 0; b--) {
            uint64_t w = p >> 5;
            if (w >= out_cap_words) return -4;
            if ((p & 31) == 0) out[w] = 0;
            uint32_t bit = (uint32_t)((code[s] >> b) & 1u);
            out[w] |= bit << (31 - (p & 31));
            p++;
        }
    }
    chunk_bit_offset[c] = p;
    *total_bits = p;
    return 0;
}

/* ----------------------------------------------------------- typed units */

/*
 * Codewords in input order, most significant bit first, into an array of
 * W-bit units (the typed data cells of Sec. IV-C, W in {8, 16, 32}); bit W-1
 * of unit 0 is stream bit 0.  aligned = 0: one dense stream, offs[c] = stream
 * bit of symbol c * 2^chunk_log2, total = bits.  aligned = 1: the gathered
 * chunks keep their own units (Sec. VI: the chunks before the optional dense
 * gathering): chunk c starts at unit offs[c], its last unit is zero-padded,
 * the final entry and total / W are the stream's units.  out holds cap_units
 * units of W bits (a uint8, uint16 or uint32 array).
 */
static void put_unit_bit(void *out, int W, uint64_t p, uint32_t bit)
{
    uint64_t u = p / (uint64_t)W;
    uint32_t k = (uint32_t)(W - 1 - (int)(p % (uint64_t)W));
    if (W == 8) ((uint8_t *)out)[u] |= (uint8_t)(bit << k);
    else if (W == 16) ((uint16_t *)out)[u] |= (uint16_t)(bit << k);
    else ((uint32_t *)out)[u] |= bit << k;
}

static void zero_unit(void *out, int W, uint64_t u)
{
    if (W == 8) ((uint8_t *)out)[u] = 0;
    else if (W == 16) ((uint16_t *)out)[u] = 0;
    else ((uint32_t *)out)[u] = 0;
}

int oracle_encode_format(const void *sym, uint64_t n, int width, const uint64_t *code, const uint8_t *len,
                         uint32_t nbins, int chunk_log2, int word_bits, int aligned, void *out,
                         uint64_t cap_units, uint64_t *offs, uint64_t *total_bits)
{
    const int W = word_bits;
    if (chunk_log2 < 0 || chunk_log2 > 40 || (W != 8 && W != 16 && W != 32) || (aligned != 0 && aligned != 1))
        return -1;
    uint64_t chunk = 1ull << chunk_log2;
    uint64_t p = 0, c = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (i % chunk == 0) {
            if (aligned) p = (p + (uint64_t)W - 1) / (uint64_t)W * (uint64_t)W;   /* next unit boundary */
            offs[c++] = aligned ? p / (uint64_t)W : p;
        }
        uint32_t s = load_sym(sym, i, width);
        if (s >= nbins) return -2;
        uint32_t l = len[s];
        if (l == 0) return -3;
        for (int b = (int)l - 1; b >= 0; b--) {
            if (p / (uint64_t)W >= cap_units) return -4;
            if (p % (uint64_t)W == 0) zero_unit(out, W, p / (uint64_t)W);
            put_unit_bit(out, W, p, (uint32_t)((code[s] >> b) & 1u));
            p++;
        }
    }
    if (aligned) p = (p + (uint64_t)W - 1) / (uint64_t)W * (uint64_t)W;
    offs[c] = aligned ? p / (uint64_t)W : p;
    *total_bits = p;
    return 0;
}

/* ------------------------------------------------------------------- decode */

/*
 * Treeless canonical decoding (Sec. IV-B2): read bits into v until v is at
 * least first[l]; the symbol is sorted_syms[entry[l] + v - first[l]].
 */
int oracle_decode(const uint32_t *stream, uint64_t total_bits, uint64_t n, const uint64_t *first,
                  const uint32_t *entry, const uint32_t *count, const uint32_t *sorted_syms,
                  uint32_t max_len, int width, void *out)
{
    uint64_t p = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t v = 0;
        uint32_t l = 0;
        for (;;) {
            if (p >= total_bits || l >= max_len) return -6;
            uint32_t bit = (stream[p >> 5] >> (31 - (p & 31))) & 1u;
            p++;
            v = 2 * v + bit;
            l++;
            if (v >= first[l]) break;
        }
        if (v - first[l] >= count[l]) return -6;
        uint32_t s = sorted_syms[entry[l] + (v - first[l])];
        if (width == 1) ((uint8_t *)out)[i] = (uint8_t)s;
        else if (width == 2) ((uint16_t *)out)[i] = (uint16_t)s;
        else ((uint32_t *)out)[i] = s;
    }
    return p == total_bits ? 0 : -6;
}
