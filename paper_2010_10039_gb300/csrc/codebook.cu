// Codebook construction (Sec. IV-B, Algorithm 1) in one CTA.
//
// GenerateCL.  The paper runs the parallel construction of Ostadzadeh et al.:
// every round makes t from the two lightest nodes, selects the leaves lighter
// than t, merges them with the waiting joined nodes (Merge Path) and melds
// adjacent pairs.  Here one round does the same with a tie rule that makes the
// result identical to the serial two-queue construction (leaves ordered by
// (count, id), a leaf before a joined node of equal weight, joined nodes in
// creation order):
//   S      = the waiting leaves and joined nodes in that order (a stable
//            leaf-first merge of two sorted queues),
//   t      = weight(S0) + weight(S1),
//   k      = number of nodes in S of weight <= t,
//   m      = k rounded down to even,
//   meld S[2j] with S[2j+1] for j < m/2, appending the results in order j.
// Every node of weight <= t leaves the queues before the node S0+S1 in the
// serial order (equal-weight leaves win the tie, equal-weight joined nodes
// are older), and the pairs leave two by two, so the serial construction melds
// exactly these pairs; an odd k leaves S[k-1] to pair with S0+S1 next round.
// The paper's sync-separated parallel regions become __syncthreads() of one
// 1024-thread CTA; the merge ranks each node by binary search in the other
// queue (the stable form of Merge Path's co-ranking).
//
// Lengths.  Instead of walking every leaf to its leader each round
// (UpdateLeafNode), each meld records the parent of its two inputs; one pass
// over the rounds in reverse gives every joined node its depth, and a leaf's
// length is its parent's depth plus one.
//
// GenerateCW + canonisation (Sec. IV-B2).  Code lengths are counted per
// length; First is filled from the longest length down so that a shorter
// codeword is numerically larger than the prefixes of longer ones; codewords of
// one length are consecutive in ascending symbol id (a warp-match rank inside
// each 1024-id slice plus a per-length running base).  Entry and the
// (length, id)-sorted symbol list form the reverse codebook.
#include "kernels.cuh"

namespace huff {

constexpr int kCbThreads = 1024;
constexpr uint32_t kCbSmemBins = 4096;     // arrays live in shared memory up to this alphabet

struct CbArrays {
    uint64_t *keys;     // P       sort keys (count << 16 | id), unused = ~0
    uint32_t *wL;       // m       leaf weights (sorted)
    uint32_t *wI;       // m       joined-node weights (creation order)
    uint32_t *parent;   // 2m      parent node id of every node
    uint32_t *temp;     // m       merged order of this round (node ids)
    uint32_t *rstart;   // m       first joined node of each round
    uint32_t *depthI;   // m       depth of joined nodes
    uint8_t *lenS;      // nbins   length by symbol id
};

__host__ __device__ inline uint32_t pow2_ceil(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t cb_array_bytes(uint32_t nbins) {
    size_t P = pow2_ceil(nbins);
    return align16(P * 8) + 6 * align16((size_t)nbins * 4) + align16((size_t)nbins * 8) + align16(nbins);
}

__device__ inline CbArrays cb_carve(uint8_t *p, uint32_t nbins) {
    CbArrays a;
    size_t P = pow2_ceil(nbins);
    a.keys = reinterpret_cast<uint64_t *>(p); p += align16(P * 8);
    a.wL = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 4);
    a.wI = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 4);
    a.parent = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 8);
    a.temp = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 4);
    a.rstart = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 4);
    a.depthI = reinterpret_cast<uint32_t *>(p); p += align16((size_t)nbins * 4);
    a.lenS = p;
    return a;
}

// Bitonic stages of stride j < 32 for the keys this thread holds (element
// e = tid + r * kCbThreads; the partner e ^ j is in the same warp, so the
// exchange is a shuffle, not a barrier-separated pass).
__device__ __forceinline__ uint64_t bitonic_warp_stages(uint64_t x, uint32_t e, uint32_t k, uint32_t jmax) {
    for (uint32_t j = jmax; j > 0; j >>= 1) {
        const uint64_t y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
        const bool up = (e & k) == 0, lower = (e & j) == 0;
        x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
    }
    return x;
}

// index of the first element > t in sorted w[lo, hi), one warp cooperating
__device__ uint32_t warp_upper_bound(const uint32_t *w, uint32_t lo, uint32_t hi, uint32_t t) {
    const uint32_t lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        uint32_t step = (hi - lo + 31) / 32;
        uint32_t pos = lo + lane * step;
        bool pred = pos < hi && w[pos] <= t;
        uint32_t cnt = __popc(__ballot_sync(0xFFFFFFFFu, pred));
        if (cnt == 0) return lo;
        uint32_t nlo = lo + (cnt - 1) * step + 1;
        uint32_t nhi = lo + cnt * step;
        if (nhi > hi) nhi = hi;
        lo = nlo;
        hi = nhi;
    }
    bool pred = lo + lane < hi && w[lo + lane] <= t;
    return lo + __popc(__ballot_sync(0xFFFFFFFFu, pred));
}

// number of elements in sorted w[lo, hi) that are < t (strict) or <= t
template <bool STRICT>
__device__ __forceinline__ uint32_t count_below(const uint32_t *w, uint32_t lo, uint32_t hi, uint32_t t) {
    uint32_t a = lo, b = hi;
    while (a < b) {
        uint32_t mid = (a + b) >> 1;
        bool go = STRICT ? (w[mid] < t) : (w[mid] <= t);
        if (go) a = mid + 1; else b = mid;
    }
    return a - lo;
}

// Builds the codebook of one histogram with the whole CTA; `arrays` holds the
// construction's arrays (shared memory for small alphabets).
__device__ __forceinline__ void codebook_body(const CbArgs &g, uint8_t *arrays) {
    __shared__ uint64_t s_sum, s_tbits;
    __shared__ uint32_t s_m, s_c, s_ih, s_it, s_mL, s_mI, s_rounds, s_maxlen, s_bad;
    __shared__ uint32_t s_count[HUFF_MAX_LEN + 1];
    __shared__ uint32_t s_base[HUFF_MAX_LEN + 1];
    __shared__ uint64_t s_first[HUFF_MAX_LEN + 1];
    __shared__ uint32_t s_entry[HUFF_MAX_LEN + 1];
    __shared__ uint32_t s_wcnt[kCbThreads / 32][HUFF_MAX_LEN + 1];

    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nbins = g.nbins;
    const uint32_t P = pow2_ceil(nbins);
    CbArrays A = cb_carve(arrays, nbins);
    huff_codebook_header *hdr = reinterpret_cast<huff_codebook_header *>(g.book);
    uint64_t *cw = reinterpret_cast<uint64_t *>(g.book + cb_cw_offset());
    uint32_t *sorted_syms = reinterpret_cast<uint32_t *>(g.book + cb_sorted_offset(nbins));

    if (tid == 0) { s_sum = 0; s_tbits = 0; s_m = 0; s_bad = 0; s_maxlen = 0; }
    if (tid <= HUFF_MAX_LEN) { s_count[tid] = 0; s_base[tid] = 0; s_first[tid] = 0; s_entry[tid] = 0; }
    __syncthreads();

    // ---- keys, used count, histogram sum
    uint64_t part = 0;
    uint32_t used = 0;
    for (uint32_t i = tid; i < P; i += kCbThreads) {
        uint64_t key = ~0ull;
        if (i < nbins) {
            uint32_t c = g.hist[i];
            part += c;
            if (c) { key = ((uint64_t)c << 16) | i; used++; }
            A.lenS[i] = 0;
            cw[i] = 0;
        }
        A.keys[i] = key;
    }
    for (int o = 16; o; o >>= 1) {
        part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        used += __shfl_xor_sync(0xFFFFFFFFu, used, o);
    }
    if (lane == 0) { atomicAdd((unsigned long long *)&s_sum, (unsigned long long)part); atomicAdd(&s_m, used); }
    __syncthreads();
    const bool overflow = s_sum >= (1ull << 32);
    const uint32_t m = overflow ? 0 : s_m;
    if (overflow && tid == 0) set_error(g.status, HUFF_ERR_HIST_OVERFLOW);

    if (m >= 2) {
        // ---- bitonic sort of the keys (ascending: count, then id; unused last).
        // Passes of stride >= 32 exchange through shared memory with a barrier
        // each; for every k, all strides below 32 run as warp shuffles in one
        // pass over the thread's elements.
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j >= 32; j >>= 1) {
                for (uint32_t i = tid; i < P / 2; i += kCbThreads) {
                    uint32_t lo = 2 * i - (i & (j - 1));
                    uint32_t hi = lo + j;
                    uint64_t x = A.keys[lo], y = A.keys[hi];
                    bool up = (lo & k) == 0;
                    if ((x > y) == up) { A.keys[lo] = y; A.keys[hi] = x; }
                }
                __syncthreads();
            }
            const uint32_t jmax = (k >> 1) < 16 ? (k >> 1) : 16;
            if (P >= 32) {
                for (uint32_t e = tid; e < P; e += kCbThreads)
                    A.keys[e] = bitonic_warp_stages(A.keys[e], e, k, jmax);
            } else {
                // fewer keys than a warp: pad the shuffle partners with the largest key
                const uint32_t e = tid;
                if (warp == 0) {
                    uint64_t x = e < P ? A.keys[e] : ~0ull;
                    x = bitonic_warp_stages(x, e, k, jmax);
                    if (e < P) A.keys[e] = x;
                }
            }
            __syncthreads();
        }
        for (uint32_t i = tid; i < m; i += kCbThreads) A.wL[i] = (uint32_t)(A.keys[i] >> 16);
        if (tid == 0) { s_c = 0; s_ih = 0; s_it = 0; s_rounds = 0; }
        __syncthreads();

        // ---- GenerateCL rounds
        for (;;) {
            const uint32_t c = s_c, ih = s_ih, it = s_it;
            if ((m - c) + (it - ih) < 2) break;
            if (warp == 0) {
                // the two lightest nodes, leaf first on equal weight
                uint32_t pc = c, pi = ih;
                uint64_t t = 0;
                for (int q = 0; q < 2; q++) {
                    bool leaf = pc < m && (pi >= it || A.wL[pc] <= A.wI[pi]);
                    t += leaf ? A.wL[pc++] : A.wI[pi++];
                }
                const uint32_t tt = (uint32_t)t;   // the total is < 2^32
                uint32_t kL = warp_upper_bound(A.wL, c, m, tt) - c;
                uint32_t kI = warp_upper_bound(A.wI, ih, it, tt) - ih;
                if ((kL + kI) & 1) {
                    // drop the last node of the merged order: a joined node wins ties for last
                    bool dropI = kI > 0 && (kL == 0 || A.wI[ih + kI - 1] >= A.wL[c + kL - 1]);
                    if (dropI) kI--; else kL--;
                }
                if (lane == 0) { s_mL = kL; s_mI = kI; }
            }
            __syncthreads();
            const uint32_t mL = s_mL, mI = s_mI;
            // stable leaf-first merge by ranking each node in the other queue
            for (uint32_t a = tid; a < mL; a += kCbThreads) {
                uint32_t r = a + count_below<true>(A.wI, ih, ih + mI, A.wL[c + a]);
                A.temp[r] = c + a;
            }
            for (uint32_t b = tid; b < mI; b += kCbThreads) {
                uint32_t r = b + count_below<false>(A.wL, c, c + mL, A.wI[ih + b]);
                A.temp[r] = m + ih + b;
            }
            __syncthreads();
            const uint32_t pairs = (mL + mI) >> 1;
            for (uint32_t j = tid; j < pairs; j += kCbThreads) {
                uint32_t x = A.temp[2 * j], y = A.temp[2 * j + 1];
                uint32_t wx = x < m ? A.wL[x] : A.wI[x - m];
                uint32_t wy = y < m ? A.wL[y] : A.wI[y - m];
                A.wI[it + j] = wx + wy;
                A.parent[x] = m + it + j;
                A.parent[y] = m + it + j;
            }
            if (tid == 0) {
                A.rstart[s_rounds] = it;
                s_rounds++;
                s_c = c + mL;
                s_ih = ih + mI;
                s_it = it + pairs;
            }
            __syncthreads();
        }

        // ---- depths: rounds in reverse (a parent is always made in a later round)
        const uint32_t nI = m - 1, rounds = s_rounds;
        if (tid == 0) A.depthI[nI - 1] = 0;
        __syncthreads();
        for (int r = (int)rounds - 1; r >= 0; r--) {
            uint32_t j0 = A.rstart[r];
            uint32_t j1 = (r + 1 < (int)rounds) ? A.rstart[r + 1] : nI;
            for (uint32_t j = j0 + tid; j < j1; j += kCbThreads)
                if (j != nI - 1) A.depthI[j] = A.depthI[A.parent[m + j] - m] + 1;
            __syncthreads();
        }
        uint32_t bad = 0;
        for (uint32_t v = tid; v < m; v += kCbThreads) {
            uint32_t d = A.depthI[A.parent[v] - m] + 1;
            if (d > HUFF_MAX_LEN) { bad = 1; d = HUFF_MAX_LEN; }
            A.lenS[(uint32_t)(A.keys[v] & 0xFFFF)] = (uint8_t)d;
        }
        if (bad) s_bad = 1;
    } else if (m == 1) {
        for (uint32_t i = tid; i < nbins; i += kCbThreads)
            if (g.hist[i]) A.lenS[i] = 1;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) set_error(g.status, HUFF_ERR_HIST_OVERFLOW);
        for (uint32_t i = tid; i < nbins; i += kCbThreads) A.lenS[i] = 0;
        __syncthreads();
    }

    // ---- canonical codewords, First, Entry, reverse codebook
    uint64_t tb = 0;
    for (uint32_t i = tid; i < nbins; i += kCbThreads) {
        uint32_t l = A.lenS[i];
        if (l) {
            atomicAdd(&s_count[l], 1u);
            tb += (uint64_t)l * g.hist[i];
        }
    }
    for (int o = 16; o; o >>= 1) tb += __shfl_xor_sync(0xFFFFFFFFu, tb, o);
    if (lane == 0 && tb) atomicAdd((unsigned long long *)&s_tbits, (unsigned long long)tb);
    __syncthreads();
    if (tid == 0) {
        uint32_t maxl = 0;
        for (uint32_t l = 1; l <= HUFF_MAX_LEN; l++) if (s_count[l]) maxl = l;
        s_maxlen = maxl;
        if (maxl) {
            s_first[maxl] = 0;
            for (int l = (int)maxl - 1; l >= 1; l--) s_first[l] = (s_first[l + 1] + s_count[l + 1] + 1) >> 1;
        }
        s_entry[1] = 0;
        for (uint32_t l = 1; l < HUFF_MAX_LEN; l++) s_entry[l + 1] = s_entry[l] + s_count[l];
    }
    __syncthreads();
    for (uint32_t base = 0; base < nbins; base += kCbThreads) {
        for (uint32_t i = tid; i < (kCbThreads / 32) * (HUFF_MAX_LEN + 1); i += kCbThreads)
            (&s_wcnt[0][0])[i] = 0;
        __syncthreads();
        const uint32_t id = base + tid;
        const uint32_t l = id < nbins ? A.lenS[id] : 0;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, l);
        const uint32_t rank_w = __popc(peers & ((1u << lane) - 1));
        if (rank_w == 0) s_wcnt[warp][l] = __popc(peers);
        __syncthreads();
        if (tid >= 1 && tid <= HUFF_MAX_LEN) {
            uint32_t off = s_base[tid];
            for (int w = 0; w < kCbThreads / 32; w++) {
                uint32_t c = s_wcnt[w][tid];
                s_wcnt[w][tid] = off;
                off += c;
            }
            s_base[tid] = off;
        }
        __syncthreads();
        if (l) {
            uint32_t rank = s_wcnt[warp][l] + rank_w;
            cw[id] = (s_first[l] + rank) | ((uint64_t)l << HUFF_CW_LEN_SHIFT);
            sorted_syms[s_entry[l] + rank] = id;
        }
        __syncthreads();
    }
    if (tid == 0) {
        hdr->nbins = nbins;
        hdr->max_len = s_maxlen;
        uint32_t nu = 0;
        for (uint32_t l = 1; l <= HUFF_MAX_LEN; l++) nu += s_count[l];
        hdr->nused = nu;
        hdr->status = overflow || s_bad ? HUFF_ERR_HIST_OVERFLOW : HUFF_OK;
        hdr->total_bits = overflow || s_bad ? 0 : s_tbits;
        hdr->nsymbols = overflow || s_bad ? 0 : s_sum;
    }
    if (tid <= HUFF_MAX_LEN) {
        hdr->first[tid] = s_first[tid];
        hdr->entry[tid] = s_entry[tid];
        hdr->count[tid] = s_count[tid];
    }
}

__global__ void __launch_bounds__(kCbThreads, 1) codebook_kernel(CbArgs g) {
    extern __shared__ __align__(16) uint8_t smem[];
    codebook_body(g, g.nbins <= kCbSmemBins ? smem : g.scratch);
}

// Codebooks of a batch: CTA b builds those of fields b, b + grid, ...;
// alphabets above the shared-memory limit use scratch + b * scratch_stride.
__global__ void __launch_bounds__(kCbThreads, 1) codebook_batch_kernel(const CbArgs *gs, uint32_t nfields,
                                                                     uint8_t *scratch, size_t scratch_stride) {
    extern __shared__ __align__(16) uint8_t smem[];
    for (uint32_t f = blockIdx.x; f < nfields; f += gridDim.x) {
        const CbArgs g = gs[f];
        codebook_body(g, g.nbins <= kCbSmemBins ? smem : scratch + blockIdx.x * scratch_stride);
        __syncthreads();     // the next field reuses the shared state
    }
}

size_t codebook_array_bytes(uint32_t nbins) { return cb_array_bytes(nbins); }

// Shared memory a batched codebook launch needs when its largest alphabet is max_nbins.
size_t codebook_batch_smem(uint32_t max_nbins) { return max_nbins <= kCbSmemBins ? cb_array_bytes(max_nbins) : 0; }

huff_status codebook_batch_prepare(uint32_t max_nbins, int *ctas_per_sm) {
    const size_t smem = codebook_batch_smem(max_nbins);
    if (!allow_dynamic_smem((const void *)codebook_batch_kernel, smem))
        return HUFF_ERR_CUDA;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, codebook_batch_kernel, kCbThreads, smem);
    *ctas_per_sm = occ < 1 ? 1 : occ;
    return HUFF_OK;
}

huff_status codebook_batch_launch(const CbArgs *d_args, uint32_t nfields, uint32_t max_nbins, uint32_t grid,
                                  uint8_t *scratch, size_t scratch_stride, cudaStream_t st) {
    codebook_batch_kernel<<<grid, kCbThreads, codebook_batch_smem(max_nbins), st>>>(d_args, nfields, scratch,
                                                                                     scratch_stride);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

size_t codebook_scratch_bytes(uint32_t nbins) {
    return nbins <= kCbSmemBins ? 0 : cb_array_bytes(nbins);
}

huff_status codebook_launch(const uint32_t *d_hist, uint32_t nbins, void *d_codebook, uint8_t *scratch,
                            uint32_t *status, cudaStream_t st) {
    CbArgs a;
    a.hist = d_hist;
    a.nbins = nbins;
    a.book = static_cast<uint8_t *>(d_codebook);
    a.scratch = scratch;
    a.status = status;
    size_t smem = nbins <= kCbSmemBins ? cb_array_bytes(nbins) : 0;
    if (!allow_dynamic_smem((const void *)codebook_kernel, smem))
        return HUFF_ERR_CUDA;
    codebook_kernel<<<1, kCbThreads, smem, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

}  // namespace huff
