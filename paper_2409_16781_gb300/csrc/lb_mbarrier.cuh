// lb_mbarrier.cuh -- shared-memory mbarrier and bulk-copy helpers (inline
// PTX for sm_103a) used by the TMA pipeline step kernels and by the
// bounded-wait self-test: barrier initialisation, arrivals with expected
// transaction bytes, a bounded parity wait, and cp.async.bulk global ->
// shared copies that complete on a barrier.
#pragma once

#include <stdint.h>

namespace lbgb {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase of parity `parity` to complete: gives up (and
// returns false) after deadline_ns of %globaltimer time or 2^24 polls,
// whichever comes first, so that a copy or an arrival that never happens
// makes the kernel report instead of hanging.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t deadline_ns = 2000000000ull) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > deadline_ns) return false;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

}  // namespace lbgb
