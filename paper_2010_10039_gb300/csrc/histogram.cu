// Histogram (Sec. IV-A; Table I rows "blockwise reduction" and "gridwise
// reduction").  The paper follows Gomez-Luna et al.: every block keeps one or
// more replicas of the histogram in shared memory, updates them with shared
// atomics and finally folds the replicas into the global histogram.
//
// GB300 form: a persistent grid streams the input in CTA-contiguous 16 KB
// rounds; each thread issues two independent 16-byte loads per round, so the
// ~6.8 TB/s of HBM3e sees enough bytes in flight with two CTAs per SM.  Each
// warp counts into its own replica (same-bin conflicts stay inside one warp),
// the replicas are folded once per CTA and only nonzero bins reach the global
// histogram.  Alphabets too large for 32-bit counters in shared memory use
// packed 16-bit counters (bins k and k + 32768 share a word) that are flushed
// to the global histogram before any of them can wrap.
#include "common.cuh"

namespace huff {

constexpr int kHistThreads = 512;
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
template <bool PACKED>
__device__ __forceinline__ void count_one(uint32_t *h, uint32_t s, uint32_t mask, uint32_t &seen) {
    seen |= s;
    if (PACKED) atomicAdd(h + (s & (kPackedWords - 1)), 1u << (((s & mask) >> 15) << 4));
    else atomicAdd(h + (s & mask), 1u);
}

template <typename Sym, bool PACKED>
__device__ __forceinline__ void count_vec(uint32_t *h, const uint4 &v, uint32_t mask, uint32_t &seen) {
#pragma unroll
    for (int j = 0; j < SymVec<Sym>::N; j++) count_one<PACKED>(h, SymVec<Sym>::get(v, j), mask, seen);
}

// Folds the shared-memory counts into the global histogram; counts in slots
// at or past nbins are symbols out of range: they set *bad and are dropped.
template <bool PACKED>
__device__ void hist_flush(uint32_t *hsm, const HistArgs &a, uint32_t &bad) {
    if (PACKED) {
        for (uint32_t w = threadIdx.x; w < kPackedWords; w += blockDim.x) {
            uint32_t v = hsm[w];
            if (v) {
                if (v & 0xFFFFu) {
                    if (w < a.nbins) atomicAdd(a.hist + w, v & 0xFFFFu); else bad = 1;
                }
                if (v >> 16) {
                    if (w + kPackedWords < a.nbins) atomicAdd(a.hist + w + kPackedWords, v >> 16); else bad = 1;
                }
                hsm[w] = 0;
            }
        }
    } else {
        for (uint32_t k = threadIdx.x; k <= a.mask; k += blockDim.x) {
            uint32_t sum = 0;
            for (uint32_t r = 0; r < a.nrep; r++) sum += hsm[r * a.stride + k];
            if (sum) {
                if (k < a.nbins) atomicAdd(a.hist + k, sum); else bad = 1;
            }
        }
    }
}

template <typename Sym, bool PACKED>
__global__ void __launch_bounds__(kHistThreads, 2) hist_kernel(HistArgs a) {
    extern __shared__ __align__(16) uint32_t hsm[];
    const uint32_t words = PACKED ? kPackedWords : a.nrep * a.stride;
    const uint32_t mask = a.mask;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) hsm[i] = 0;
    __syncthreads();
    uint32_t *my = PACKED ? hsm : hsm + ((threadIdx.x >> 5) % a.nrep) * a.stride;
    uint32_t seen = 0, bad = 0;

    const uint4 *vec = reinterpret_cast<const uint4 *>(a.base + a.head * sizeof(Sym));
    constexpr uint64_t kRound = 2ull * kHistThreads;              // vectors per CTA round
    constexpr uint32_t kSymsPerRound = kRound * SymVec<Sym>::N;
    // packed counters: flush before any 16-bit field can reach 65536
    constexpr uint32_t kRoundsPerEpoch = PACKED ? 65535u / kSymsPerRound : 0xFFFFFFFFu;
    const uint64_t nrounds = (a.nvec + kRound - 1) / kRound;
    uint32_t since = 0;
    for (uint64_t r = blockIdx.x; r < nrounds; r += gridDim.x) {
        const uint64_t i0 = r * kRound + threadIdx.x, i1 = i0 + kHistThreads;
        if (i1 < a.nvec) {
            uint4 v0 = vec[i0], v1 = vec[i1];
            count_vec<Sym, PACKED>(my, v0, mask, seen);
            count_vec<Sym, PACKED>(my, v1, mask, seen);
        } else if (i0 < a.nvec) {
            count_vec<Sym, PACKED>(my, vec[i0], mask, seen);
        }
        if (PACKED && ++since == kRoundsPerEpoch) {
            __syncthreads();
            hist_flush<true>(hsm, a, bad);
            __syncthreads();
            since = 0;
        }
    }
    if (PACKED) {
        __syncthreads();
        hist_flush<true>(hsm, a, bad);
        __syncthreads();
    }
    // head (before the first aligned address) and tail (after the last whole vector)
    const uint64_t tail0 = a.head + a.nvec * SymVec<Sym>::N;
    const Sym *sp = reinterpret_cast<const Sym *>(a.base);
    const uint64_t nrest = a.head + (a.n - tail0);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nrest; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t idx = i < a.head ? i : tail0 + (i - a.head);
        count_one<PACKED>(my, sp[idx], mask, seen);
    }
    __syncthreads();
    hist_flush<PACKED>(hsm, a, bad);
    if (bad || seen > mask) set_error(a.status, HUFF_ERR_SYMBOL_RANGE);
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
    const bool packed = nbins > 16384;
    uint32_t slots = 1;
    while (slots < nbins) slots <<= 1;
    a.mask = slots - 1;
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
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return HUFF_ERR_CUDA;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kHistThreads, smem);
    if (occ < 1) occ = 1;
    uint64_t rounds = (a.nvec + 2 * kHistThreads - 1) / (2 * kHistThreads);
    uint64_t grid = (uint64_t)sm_count() * occ;
    if (grid > rounds) grid = rounds;
    if (grid < 1) grid = 1;
    if (cudaMemsetAsync(d_hist, 0, nbins * sizeof(uint32_t), st) != cudaSuccess) return HUFF_ERR_CUDA;
    kern<<<(unsigned)grid, kHistThreads, smem, st>>>(a);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
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
