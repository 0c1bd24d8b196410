// Shared device helpers for libhuff (sm_103a): status word, bulk-copy (TMA)
// staging with mbarriers, and small warp/block utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "huff.h"

namespace huff {

constexpr int kWsHeaderBytes = 256;          // status word + call scratch header
constexpr uint32_t kSpinLimit = 1u << 22;    // polls before a device wait gives up

struct WsHeader {
    uint32_t status;      // sticky first error (huff_status)
    uint32_t pad0;
    uint64_t pad[31];
};

// Scratch of one encode call, after the header.
struct EncodeScratch {
    uint32_t tile_counter;
    uint32_t pad;
};

__device__ __forceinline__ void set_error(uint32_t *status, uint32_t code) {
    atomicCAS(status, 0u, code);
}

__device__ __forceinline__ uint64_t cw_code(uint64_t cw) { return cw & ((1ull << HUFF_CW_LEN_SHIFT) - 1); }
__device__ __forceinline__ uint32_t cw_len(uint64_t cw) { return (uint32_t)(cw >> HUFF_CW_LEN_SHIFT); }

__host__ __device__ inline size_t cb_cw_offset() { return sizeof(huff_codebook_header); }
__host__ __device__ inline size_t cb_sorted_offset(uint32_t nbins) {
    return sizeof(huff_codebook_header) + 8ull * nbins;
}

// ---------------------------------------------------------------- mbarrier + bulk copy

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// One-dimensional bulk copy global -> shared (the non-tensor TMA form).
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Waits for phase `parity` of `bar`, suspended in hardware for up to
// hint_ns (the thread resumes as soon as the phase completes).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns) : "memory");
    return ok != 0;
}

constexpr uint32_t kWaitHintNs = 100000;         // suspend up to 0.1 ms per attempt
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // a device wait gives up after 2 s

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of `bar`; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity, kWaitHintNs)) return true;
    const uint64_t t0 = global_ns();
    while (global_ns() - t0 < kWaitLimitNs)
        if (mbar_try_wait(bar, parity, kWaitHintNs)) return true;
    return false;
}

// ---------------------------------------------------------------- global flag access

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------- host-side helpers

int sm_count();                       // cached multiprocessor count of the current device
// Lets `func` use up to the device's opt-in maximum of dynamic shared memory
// (once per function and device).  The limit is never lowered again, so
// launches of the same kernel with different sizes -- from other threads,
// other plans or captured graphs -- cannot invalidate each other; false if
// `need` is above the maximum or the call failed.
bool allow_dynamic_smem(const void *func, size_t need);
void note_launch(int k = 1);          // launch counter for huff_launch_count()

}  // namespace huff
