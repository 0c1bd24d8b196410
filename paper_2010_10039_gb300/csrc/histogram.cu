// Histogram (Sec. IV-A; Table I rows "blockwise reduction" and "gridwise
// reduction").  The paper follows Gomez-Luna et al.: every block keeps one or
// more replicas of the histogram in shared memory, updates them with shared
// atomics and finally folds the replicas into the global histogram.
//
// GB300 form: a persistent grid streams the input in CTA-contiguous 16 KB
// rounds; each thread issues two independent 16-byte loads per round, and
// loads the next round's pair before it counts the current one.  Each
// warp counts into its own replica (same-bin conflicts stay inside one warp),
// the replicas are folded once per CTA and only nonzero bins reach the global
// histogram.  Alphabets too large for 32-bit counters in shared memory use
// packed 16-bit counters (bins k and k + 32768 share a word).  The increment
// that takes a counter to 0x8000 moves 0x8000 to the global bin; with a
// barrier every 32,768 symbols of the CTA, every counter is at most 0x7FFF at
// each barrier, so none can pass 0xFFFF in between, and the table is folded
// into the global histogram once, at the end.
#include "kernels.cuh"

namespace huff {

constexpr int kHistThreads = 512;
constexpr int kHistPackedThreads = 1024;      // the packed table fills one CTA per SM: give it more warps

__host__ __device__ constexpr int hist_threads(bool packed) { return packed ? kHistPackedThreads : kHistThreads; }
constexpr uint32_t kPackedWords = 32768;       // 65536 16-bit counters

template <typename Sym>
struct SymVec;
template <>
struct SymVec<uint8_t> {
    static constexpr int N = 16;
    __device__ __forceinline__ static uint32_t get(const uint4 &v, int j) {
        uint32_t w = (j < 4) ? v.x : (j < 8) ? v.y : (j < 12) ? v.z : v.w;
        return (w >> (8 * (j & 3))) & 0xFFu;
    }
};
template <>
struct SymVec<uint16_t> {
    static constexpr int N = 8;
    __device__ __forceinline__ static uint32_t get(const uint4 &v, int j) {
        uint32_t w = (j < 2) ? v.x : (j < 4) ? v.y : (j < 6) ? v.z : v.w;
        return (j & 1) ? (w >> 16) : (w & 0xFFFFu);
    }
};
template <>
struct SymVec<uint32_t> {
    static constexpr int N = 4;
    __device__ __forceinline__ static uint32_t get(const uint4 &v, int j) {
        return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
    }
};

struct HistArgs {
    uint32_t nwin;            // windows of 65,536 bins (alphabets above 65,536 bins); 1 otherwise
    uint32_t pad;
    const uint8_t *base;      // first byte of the input
    uint64_t n;               // symbols
    uint64_t head;            // symbols before the first 16-byte aligned address
    uint64_t nvec;            // whole 16-byte vectors after the head
    uint32_t nbins;
    uint32_t mask;            // slots per replica - 1 (a power of two minus one, >= nbins - 1)
    uint32_t nrep;            // replicas (32-bit layout)
    uint32_t stride;          // words per replica
    uint32_t *hist;
    uint32_t *status;
};

// Counts one symbol without a branch: replicas have a power-of-two number of
// slots (mask + 1 >= nbins) and symbols are masked into them; `seen` ORs the
// symbols, so a symbol beyond the slots is caught after the loop, and one in
// [nbins, mask] leaves a count in a slot past nbins (both are range errors).
// Packed counters with CARRY: the increment that takes a 16-bit counter from
// 0x7FFF to 0x8000 (exactly one per crossing, atomics being ordered) takes
// 0x8000 back out and adds it to the global bin.  A slot at or past nbins is a
// range error (*bad); its count is dropped.
struct Carry {
    uint32_t *hist;
    uint32_t nbins;
};

template <bool PACKED, bool CARRY = false>
__device__ __forceinline__ void count_one(uint32_t *h, uint32_t s, uint32_t mask, uint32_t &seen,
                                          const Carry &cy = Carry{nullptr, 0}, uint32_t *bad = nullptr) {
    seen |= s;
    if (PACKED) {
        const uint32_t sh = ((s & mask) >> 15) << 4;
        uint32_t *w = h + (s & (kPackedWords - 1));
        if (CARRY) {
            const uint32_t old = atomicAdd(w, 1u << sh);
            if (((old >> sh) & 0xFFFFu) == 0x7FFFu) {
                atomicSub(w, 0x8000u << sh);
                if ((s & mask) < cy.nbins) atomicAdd(cy.hist + (s & mask), 0x8000u);
                else *bad = 1;
            }
        } else {
            atomicAdd(w, 1u << sh);
        }
    } else {
        atomicAdd(h + (s & mask), 1u);
    }
}

template <typename Sym, bool PACKED, bool CARRY = false>
__device__ __forceinline__ void count_vec(uint32_t *h, const uint4 &v, uint32_t mask, uint32_t &seen,
                                          const Carry &cy = Carry{nullptr, 0}, uint32_t *bad = nullptr) {
    if (PACKED && CARRY) {
        // all the vector's increments first, then the crossings: the increments
        // do not wait for one another's results (a carry only has to land
        // before the epoch's barrier)
        constexpr int N = SymVec<Sym>::N;
        uint32_t old[N], sh[N], sm[N];
#pragma unroll
        for (int j = 0; j < N; j++) {
            const uint32_t s = SymVec<Sym>::get(v, j);
            seen |= s;
            sm[j] = s & mask;
            sh[j] = (sm[j] >> 15) << 4;
            old[j] = atomicAdd(h + (s & (kPackedWords - 1)), 1u << sh[j]);
        }
#pragma unroll
        for (int j = 0; j < N; j++) {
            if (((old[j] >> sh[j]) & 0xFFFFu) == 0x7FFFu) {
                atomicSub(h + (sm[j] & (kPackedWords - 1)), 0x8000u << sh[j]);
                if (sm[j] < cy.nbins) atomicAdd(cy.hist + sm[j], 0x8000u);
                else *bad = 1;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < SymVec<Sym>::N; j++)
            count_one<PACKED, CARRY>(h, SymVec<Sym>::get(v, j), mask, seen, cy, bad);
    }
}

// Folds the shared-memory counts into the global histogram; counts in slots
// at or past nbins are symbols out of range: they set *bad and are dropped.
template <bool PACKED>
__device__ void hist_flush(uint32_t *hsm, uint32_t *hist, uint32_t nbins, uint32_t mask, uint32_t nrep,
                           uint32_t stride, uint32_t &bad) {
    if (PACKED) {
        for (uint32_t w = threadIdx.x; w < kPackedWords; w += blockDim.x) {
            uint32_t v = hsm[w];
            if (v) {
                if (v & 0xFFFFu) {
                    if (w < nbins) atomicAdd(hist + w, v & 0xFFFFu); else bad = 1;
                }
                if (v >> 16) {
                    if (w + kPackedWords < nbins) atomicAdd(hist + w + kPackedWords, v >> 16); else bad = 1;
                }
                hsm[w] = 0;
            }
        }
    } else {
        for (uint32_t k = threadIdx.x; k <= mask; k += blockDim.x) {
            uint32_t sum = 0;
            for (uint32_t r = 0; r < nrep; r++) sum += hsm[r * stride + k];
            if (sum) {
                if (k < nbins) atomicAdd(hist + k, sum); else bad = 1;
            }
        }
    }
}

template <typename Sym, bool PACKED>
__global__ void __launch_bounds__(hist_threads(PACKED), PACKED ? 1 : 2) hist_kernel(HistArgs a) {
    constexpr int T = hist_threads(PACKED);
    extern __shared__ __align__(16) uint32_t hsm[];
    const uint32_t words = PACKED ? kPackedWords : a.nrep * a.stride;
    const uint32_t mask = a.mask;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) hsm[i] = 0;
    __syncthreads();
    uint32_t *my = PACKED ? hsm : hsm + ((threadIdx.x >> 5) % a.nrep) * a.stride;
    uint32_t seen = 0, bad = 0;

    const uint4 *vec = reinterpret_cast<const uint4 *>(a.base + a.head * sizeof(Sym));
    constexpr uint64_t kRound = 2ull * T;                         // vectors per CTA round
    constexpr uint32_t kSymsPerRound = kRound * SymVec<Sym>::N;
    // packed counters: a barrier at least every 32,768 symbols of the CTA (an
    // epoch), so that a counter at most 0x7FFF at its start stays below 0x10000
    constexpr uint32_t kRoundsPerEpoch = PACKED ? 32768u / kSymsPerRound : 0xFFFFFFFFu;
    static_assert(!PACKED || kRoundsPerEpoch >= 1, "a round must fit in an epoch");
    const Carry cy{a.hist, a.nbins};
    const uint64_t nrounds = (a.nvec + kRound - 1) / kRound;
    uint32_t since = 0;
    uint4 v0 = make_uint4(0u, 0u, 0u, 0u), v1 = v0;
    if (blockIdx.x < nrounds) {
        const uint64_t i0 = blockIdx.x * kRound + threadIdx.x, i1 = i0 + T;
        if (i0 < a.nvec) v0 = vec[i0];
        if (i1 < a.nvec) v1 = vec[i1];
    }
    for (uint64_t r = blockIdx.x; r < nrounds; r += gridDim.x) {
        const uint64_t i0 = r * kRound + threadIdx.x, i1 = i0 + T;
        // the next round's vectors are loaded before this round is counted
        uint4 n0 = v0, n1 = v1;
        const uint64_t rn = r + gridDim.x;
        if (rn < nrounds) {
            const uint64_t j0 = rn * kRound + threadIdx.x, j1 = j0 + T;
            if (j0 < a.nvec) n0 = vec[j0];
            if (j1 < a.nvec) n1 = vec[j1];
        }
        if (i1 < a.nvec) {
            count_vec<Sym, PACKED, PACKED>(my, v0, mask, seen, cy, &bad);
            count_vec<Sym, PACKED, PACKED>(my, v1, mask, seen, cy, &bad);
        } else if (i0 < a.nvec) {
            count_vec<Sym, PACKED, PACKED>(my, v0, mask, seen, cy, &bad);
        }
        v0 = n0;
        v1 = n1;
        if (PACKED && ++since == kRoundsPerEpoch) {
            __syncthreads();
            since = 0;
        }
    }
    if (PACKED) __syncthreads();     // the head and tail below are an epoch of their own
    // head (before the first aligned address) and tail (after the last whole vector)
    const uint64_t tail0 = a.head + a.nvec * SymVec<Sym>::N;
    const Sym *sp = reinterpret_cast<const Sym *>(a.base);
    const uint64_t nrest = a.head + (a.n - tail0);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nrest; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t idx = i < a.head ? i : tail0 + (i - a.head);
        count_one<PACKED, PACKED>(my, sp[idx], mask, seen, cy, &bad);
    }
    __syncthreads();
    hist_flush<PACKED>(hsm, a.hist, a.nbins, a.mask, a.nrep, a.stride, bad);
    if (bad || seen > mask) set_error(a.status, HUFF_ERR_SYMBOL_RANGE);
}

// ---------------------------------------------------------------- alphabets above 65,536 bins

// The bins are split into windows of 65,536 packed counters (the most one
// CTA's shared memory holds), and the grid into nwin groups of CTAs: group w
// counts the symbols in [w * 65536, (w + 1) * 65536), reading all of the
// input, so each CTA still owns every counter it increments (hot bins
// contend only inside one CTA) and folds one window at the end.  The input
// is read nwin times; the alternative of sending each symbol to the CTA that
// owns its bin serialises the hot bins of skewed alphabets on one SM.
// Counters, carries and epochs are those of the packed 65,536-bin kernel.
template <typename Sym>
__global__ void __launch_bounds__(kHistPackedThreads, 1) hist_window_kernel(HistArgs a) {
    constexpr int T = kHistPackedThreads;
    extern __shared__ __align__(16) uint32_t hsm[];
    for (uint32_t i = threadIdx.x; i < kPackedWords; i += blockDim.x) hsm[i] = 0;
    __syncthreads();
    const uint32_t win = blockIdx.x % a.nwin, grp = blockIdx.x / a.nwin, ngrp = gridDim.x / a.nwin;
    const uint32_t lo = win << 16;
    uint32_t seen = 0, bad = 0;
    auto count = [&](uint32_t s) {
        seen |= s;
        const uint32_t d = s - lo;
        if (d < 65536u) {
            const uint32_t sh = (d >> 15) << 4;
            uint32_t *w = hsm + (d & (kPackedWords - 1));
            const uint32_t old = atomicAdd(w, 1u << sh);
            if (((old >> sh) & 0xFFFFu) == 0x7FFFu) {
                atomicSub(w, 0x8000u << sh);
                if (s < a.nbins) atomicAdd(a.hist + s, 0x8000u); else bad = 1;
            }
        }
    };
    const uint4 *vec = reinterpret_cast<const uint4 *>(a.base + a.head * sizeof(Sym));
    constexpr uint64_t kRound = 2ull * T;
    constexpr uint32_t kSymsPerRound = kRound * SymVec<Sym>::N;
    constexpr uint32_t kRoundsPerEpoch = 32768u / kSymsPerRound;
    static_assert(kRoundsPerEpoch >= 1, "a round must fit in an epoch");
    const uint64_t nrounds = (a.nvec + kRound - 1) / kRound;
    uint32_t since = 0;
    for (uint64_t r = grp; r < nrounds; r += ngrp) {
        const uint64_t i0 = r * kRound + threadIdx.x, i1 = i0 + T;
        if (i1 < a.nvec) {
            const uint4 v0 = vec[i0], v1 = vec[i1];
#pragma unroll
            for (int j = 0; j < SymVec<Sym>::N; j++) count(SymVec<Sym>::get(v0, j));
#pragma unroll
            for (int j = 0; j < SymVec<Sym>::N; j++) count(SymVec<Sym>::get(v1, j));
        } else if (i0 < a.nvec) {
            const uint4 v0 = vec[i0];
#pragma unroll
            for (int j = 0; j < SymVec<Sym>::N; j++) count(SymVec<Sym>::get(v0, j));
        }
        if (++since == kRoundsPerEpoch) {
            __syncthreads();
            since = 0;
        }
    }
    __syncthreads();
    const uint64_t tail0 = a.head + a.nvec * SymVec<Sym>::N;
    const Sym *sp = reinterpret_cast<const Sym *>(a.base);
    const uint64_t nrest = a.head + (a.n - tail0);
    for (uint64_t i = grp * (uint64_t)blockDim.x + threadIdx.x; i < nrest; i += (uint64_t)ngrp * blockDim.x)
        count(sp[i < a.head ? i : tail0 + (i - a.head)]);
    __syncthreads();
    for (uint32_t w = threadIdx.x; w < kPackedWords; w += blockDim.x) {
        const uint32_t v = hsm[w];
        if (v & 0xFFFFu) {
            if (lo + w < a.nbins) atomicAdd(a.hist + lo + w, v & 0xFFFFu); else bad = 1;
        }
        if (v >> 16) {
            if (lo + w + kPackedWords < a.nbins) atomicAdd(a.hist + lo + w + kPackedWords, v >> 16); else bad = 1;
        }
    }
    if (bad || seen > a.mask) set_error(a.status, HUFF_ERR_SYMBOL_RANGE);
}

// ---------------------------------------------------------------- batched histogram

// Every CTA counts whole tiles (CTA-strided over the tile list) into its
// replicas and folds them into the tile's field after each tile.  Tiles of a
// packed (> 16384-bin) batch hold at most 65,535 symbols, so 16-bit counters
// never wrap.
template <typename Sym, bool PACKED>
__global__ void __launch_bounds__(kHistThreads, 2) hist_batch_kernel(const HistTile *tiles, uint32_t ntiles,
                                                                      const HistField *fields, uint32_t mask,
                                                                      uint32_t nrep, uint32_t stride) {
    extern __shared__ __align__(16) uint32_t hsm[];
    constexpr int V = SymVec<Sym>::N;
    const uint32_t words = PACKED ? kPackedWords : nrep * stride;
    uint32_t *my = PACKED ? hsm : hsm + ((threadIdx.x >> 5) % nrep) * stride;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) hsm[i] = 0;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();
        const HistTile T = tiles[t];
        const HistField F = fields[T.field];
        const Sym *sp = reinterpret_cast<const Sym *>(F.sym);
        uint32_t seen = 0, bad = 0;
        // [start, a0) scalars, whole vectors from a0, then a scalar tail
        const uint64_t a0 = T.start + F.head < T.end ? T.start + F.head : T.end;
        const uint64_t nv = (T.end - a0) / V;
        const uint64_t tail0 = a0 + nv * V;
        if (threadIdx.x < a0 - T.start) count_one<PACKED>(my, sp[T.start + threadIdx.x], mask, seen);
        if (threadIdx.x < T.end - tail0) count_one<PACKED>(my, sp[tail0 + threadIdx.x], mask, seen);
        const uint4 *vec = reinterpret_cast<const uint4 *>(sp + a0);
        uint64_t i = threadIdx.x;
        for (; i + 3 * kHistThreads < nv; i += 4 * kHistThreads) {
            const uint4 v0 = vec[i], v1 = vec[i + kHistThreads], v2 = vec[i + 2 * kHistThreads],
                        v3 = vec[i + 3 * kHistThreads];
            count_vec<Sym, PACKED>(my, v0, mask, seen);
            count_vec<Sym, PACKED>(my, v1, mask, seen);
            count_vec<Sym, PACKED>(my, v2, mask, seen);
            count_vec<Sym, PACKED>(my, v3, mask, seen);
        }
        for (; i < nv; i += kHistThreads) count_vec<Sym, PACKED>(my, vec[i], mask, seen);
        __syncthreads();
        if (PACKED) {
            hist_flush<true>(hsm, F.hist, F.nbins, mask, 1, kPackedWords, bad);    // also clears the counters
        } else {
            hist_flush<false>(hsm, F.hist, F.nbins, mask, nrep, stride, bad);
            __syncthreads();
            for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) hsm[w] = 0;
        }
        if (bad || seen > mask) set_error(F.status, HUFF_ERR_SYMBOL_RANGE);
    }
}

template <typename Sym>
static huff_status launch_hist(const void *d_sym, uint64_t n, uint32_t nbins, uint32_t *d_hist,
                               uint32_t *status, cudaStream_t st) {
    HistArgs a;
    a.base = static_cast<const uint8_t *>(d_sym);
    a.n = n;
    uint64_t mis = (16 - ((uintptr_t)d_sym & 15)) & 15;
    a.head = mis / sizeof(Sym);
    if (a.head > n) a.head = n;
    a.nvec = (n - a.head) / SymVec<Sym>::N;
    a.nbins = nbins;
    a.hist = d_hist;
    a.status = status;
    a.nwin = 1;
    a.pad = 0;
    uint32_t slots = 1;
    while (slots < nbins) slots <<= 1;
    a.mask = slots - 1;
    if (nbins > 65536) {
        if (sizeof(Sym) != 4) return HUFF_ERR_INVALID_ARG;
        a.nwin = (nbins + 65535) / 65536;
        const size_t smem = kPackedWords * 4;
        if (!allow_dynamic_smem((const void *)hist_window_kernel<Sym>, smem)) return HUFF_ERR_CUDA;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hist_window_kernel<Sym>, kHistPackedThreads, smem);
        if (occ < 1) occ = 1;
        // every window gets the same number of CTAs, at least one
        uint64_t per = (uint64_t)sm_count() * occ / a.nwin;
        const uint64_t rounds = (a.nvec + 2ull * kHistPackedThreads - 1) / (2ull * kHistPackedThreads);
        if (per > rounds) per = rounds;
        if (per < 1) per = 1;
        if (cudaMemsetAsync(d_hist, 0, nbins * sizeof(uint32_t), st) != cudaSuccess) return HUFF_ERR_CUDA;
        hist_window_kernel<Sym><<<(unsigned)(per * a.nwin), kHistPackedThreads, smem, st>>>(a);
        note_launch();
        return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
    }
    const bool packed = nbins > 16384;
    size_t smem;
    if (packed) {
        a.nrep = 1;
        a.stride = kPackedWords;
        smem = kPackedWords * 4;
    } else {
        // one replica per warp, padded so one bin of different replicas hits different banks
        a.stride = slots + 1;
        const uint32_t warps = kHistThreads / 32;
        uint32_t r = (uint32_t)((100 * 1024) / (a.stride * 4ull));
        a.nrep = r > warps ? warps : (r < 1 ? 1 : r);
        smem = (size_t)a.nrep * a.stride * 4;
    }
    void (*kern)(HistArgs) = packed ? hist_kernel<Sym, true> : hist_kernel<Sym, false>;
    if (!allow_dynamic_smem((const void *)kern, smem))
        return HUFF_ERR_CUDA;
    const int threads = hist_threads(packed);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (occ < 1) occ = 1;
    uint64_t rounds = (a.nvec + 2ull * threads - 1) / (2ull * threads);
    uint64_t grid = (uint64_t)sm_count() * occ;
    if (grid > rounds) grid = rounds;
    if (grid < 1) grid = 1;
    if (cudaMemsetAsync(d_hist, 0, nbins * sizeof(uint32_t), st) != cudaSuccess) return HUFF_ERR_CUDA;
    kern<<<(unsigned)grid, threads, smem, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

// ---------------------------------------------------------------- batched launch

uint64_t histogram_batch_tile(uint32_t max_nbins) { return max_nbins > 16384 ? 32768 : 131072; }

// Replica layout of a batched launch whose largest alphabet is max_nbins.
static void batch_layout(uint32_t max_nbins, uint32_t *mask, uint32_t *nrep, uint32_t *stride, size_t *smem) {
    uint32_t slots = 1;
    while (slots < max_nbins) slots <<= 1;
    *mask = slots - 1;
    if (max_nbins > 16384) {
        *nrep = 1;
        *stride = kPackedWords;
        *smem = kPackedWords * 4;
    } else {
        *stride = slots + 1;
        const uint32_t warps = kHistThreads / 32;
        uint32_t r = (uint32_t)((100 * 1024) / (*stride * 4ull));
        *nrep = r > warps ? warps : (r < 1 ? 1 : r);
        *smem = (size_t)*nrep * *stride * 4;
    }
}

template <typename Sym>
static void (*batch_kernel(uint32_t max_nbins))(const HistTile *, uint32_t, const HistField *, uint32_t, uint32_t,
                                                 uint32_t) {
    return max_nbins > 16384 ? hist_batch_kernel<Sym, true> : hist_batch_kernel<Sym, false>;
}

template <typename Sym>
static huff_status batch_prepare(uint32_t max_nbins, int *ctas_per_sm) {
    uint32_t mask, nrep, stride;
    size_t smem;
    batch_layout(max_nbins, &mask, &nrep, &stride, &smem);
    auto kern = batch_kernel<Sym>(max_nbins);
    if (!allow_dynamic_smem((const void *)kern, smem))
        return HUFF_ERR_CUDA;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kHistThreads, smem);
    *ctas_per_sm = occ < 1 ? 1 : occ;
    return HUFF_OK;
}

template <typename Sym>
static huff_status batch_launch(const HistTile *d_tiles, uint32_t ntiles, const HistField *d_fields,
                                uint32_t max_nbins, uint32_t grid, cudaStream_t st) {
    uint32_t mask, nrep, stride;
    size_t smem;
    batch_layout(max_nbins, &mask, &nrep, &stride, &smem);
    batch_kernel<Sym>(max_nbins)<<<grid, kHistThreads, smem, st>>>(d_tiles, ntiles, d_fields, mask, nrep, stride);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

huff_status histogram_batch_prepare(huff_dtype dtype, uint32_t max_nbins, int *ctas_per_sm) {
    switch (dtype) {
        case HUFF_U8: return batch_prepare<uint8_t>(max_nbins, ctas_per_sm);
        case HUFF_U16: return batch_prepare<uint16_t>(max_nbins, ctas_per_sm);
        case HUFF_U32: return batch_prepare<uint32_t>(max_nbins, ctas_per_sm);
    }
    return HUFF_ERR_INVALID_ARG;
}

huff_status histogram_batch_launch(huff_dtype dtype, const HistTile *d_tiles, uint32_t ntiles,
                                   const HistField *d_fields, uint32_t max_nbins, uint32_t grid, cudaStream_t st) {
    switch (dtype) {
        case HUFF_U8: return batch_launch<uint8_t>(d_tiles, ntiles, d_fields, max_nbins, grid, st);
        case HUFF_U16: return batch_launch<uint16_t>(d_tiles, ntiles, d_fields, max_nbins, grid, st);
        case HUFF_U32: return batch_launch<uint32_t>(d_tiles, ntiles, d_fields, max_nbins, grid, st);
    }
    return HUFF_ERR_INVALID_ARG;
}

huff_status histogram_launch(const void *d_sym, uint64_t n, huff_dtype dtype, uint32_t nbins,
                             uint32_t *d_hist, uint32_t *status, cudaStream_t st) {
    switch (dtype) {
        case HUFF_U8: return launch_hist<uint8_t>(d_sym, n, nbins, d_hist, status, st);
        case HUFF_U16: return launch_hist<uint16_t>(d_sym, n, nbins, d_hist, status, st);
        case HUFF_U32: return launch_hist<uint32_t>(d_sym, n, nbins, d_hist, status, st);
    }
    return HUFF_ERR_INVALID_ARG;
}

}  // namespace huff
