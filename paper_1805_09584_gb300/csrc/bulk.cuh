// Shared-memory pipeline primitives (sm_100 family): mbarriers and 1-D bulk
// copies global -> shared (cp.async.bulk, completion counted in bytes on an
// mbarrier).  Every wait is bounded: it gives up after a time limit read from
// the global nanosecond timer (or when a shared stop flag is raised by another
// warp), so that a kernel whose pipeline stalls ends with an error status
// instead of spinning forever.
#pragma once

#include <stdint.h>

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity to complete.  Returns false if the wait
// gave up: after limit_ns (default ~2 s), after 2^24 polls, or when *stop becomes
// non-zero.
constexpr uint64_t MBAR_WAIT_NS = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, const volatile int *stop = nullptr,
                                          uint64_t limit_ns = MBAR_WAIT_NS) {
    if (mbar_try(a, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (int i = 1; i < (1 << 24); i++) {
        if (mbar_try(a, parity)) return true;
        if ((i & 255) == 0) {
            if (stop && *stop) return false;
            if (globaltimer_ns() - t0 > limit_ns) return false;
        }
    }
    return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
// 1-D bulk copy global -> shared: both addresses 16-byte aligned, size a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
