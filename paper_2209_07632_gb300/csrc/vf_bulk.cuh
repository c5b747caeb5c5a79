// Bulk asynchronous copies (global -> shared) completed on an mbarrier, for
// per-warp prefetch pipelines on sm_100-class GPUs (inline PTX).
//
// A copy moves a 16-byte aligned, 16-byte multiple range; callers copy the
// aligned superset of the bytes they need (so every pool the copies read
// from is padded by at least 16 bytes at its end).  Every wait is bounded:
// after `limit` polls the wait gives up and reports failure, and the kernel
// records a timeout instead of spinning.
#pragma once

#include <stdint.h>

namespace vf {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the async (bulk-copy) proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order earlier generic-proxy accesses of shared memory before later
// async-proxy writes to it (the buffer is reused)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// plain arrival (count 1), e.g. a consumer releasing a ring slot
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// non-blocking test: has the phase with the given parity completed?
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Copy the aligned superset of [src, src + bytes) to dst (16-byte aligned);
// returns the number of bytes moved and sets *pre to the offset of src
// inside dst.
__device__ __forceinline__ uint32_t bulk_superset(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                  uint32_t* pre) {
    const uintptr_t s = reinterpret_cast<uintptr_t>(src);
    const uintptr_t a = s & ~uintptr_t(15);
    const uint32_t p = (uint32_t)(s - a);
    const uint32_t len = (p + bytes + 15u) & ~15u;
    *pre = p;
    if (len) bulk_g2s(dst, reinterpret_cast<const void*>(a), len, bar);
    return len;
}

__device__ __forceinline__ uint32_t superset_len(const void* src, uint32_t bytes) {
    const uintptr_t s = reinterpret_cast<uintptr_t>(src);
    const uint32_t p = (uint32_t)(s & 15u);
    return (p + bytes + 15u) & ~15u;
}

}  // namespace vf
