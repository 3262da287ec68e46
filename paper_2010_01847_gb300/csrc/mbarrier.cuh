// mbarrier helpers shared by the kernels that wait on one: the staged kernel
// (bulk copies of the TMA engine complete on an mbarrier) and the
// cluster-resident kernel (asynchronous remote stores of the neighbouring
// CTAs complete on one).  Every wait is bounded: a wait that gives up ORs
// its bit into a device status word (read back by the host as LBM_ETIMEOUT)
// and returns false, so that the kernel can stop instead of hanging.
#pragma once

#include <stdint.h>

namespace plbm {

// Limits of a bounded wait: about 2 s at the maximum SM clock, or 2^28 polls.
constexpr long long WAIT_CYCLES = 4000000000LL;
constexpr long long WAIT_ITERS = 1LL << 28;

// Status bits a bounded wait that gives up sets.
constexpr int STATUS_STAGED = 1;      // staged kernel (bulk-copy ring)
constexpr int STATUS_RESIDENT = 2;    // cluster-resident kernel (ghost exchange)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// One poll of the phase with the given parity.  CLUSTER: acquire at cluster
// scope, for barriers that remote stores of other CTAs complete.
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    if (CLUSTER)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity: true when it completed;
// false when the wait gave up at its iteration or clock limit, after ORing
// `bit` into *status.
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *status, int bit) {
    if (mbar_try<CLUSTER>(bar, parity)) return true;
    const long long t0 = clock64();
    for (long long it = 0; it < WAIT_ITERS; ++it) {
        if (mbar_try<CLUSTER>(bar, parity)) return true;
        if ((it & 255) == 255 && clock64() - t0 > WAIT_CYCLES) break;
    }
    atomicOr(status, bit);
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

}  // namespace plbm
