// Device helpers shared by the two Chamfer kernels: the status word, a prefix search, a
// three-input minimum, and bulk copies into shared memory behind mbarriers whose waits are
// all bounded (a wait that gives up lets the kernel report DC_ETIMEOUT and return).
#pragma once

#include <stdint.h>

#include "dc_internal.cuh"

namespace dc {
namespace {

typedef unsigned long long u64;

__device__ __forceinline__ void set_status(int* st, int code) { atomicCAS(st, DC_OK, code); }

__device__ __forceinline__ int last_le(const int* pre, int n, int g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---- three-input minimum (one instruction on sm_100+) ----
__device__ __forceinline__ float min3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ---- mbarrier + bulk copy (global -> shared), all waits bounded ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(u64* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, u64* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try(u64* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ u64 globaltimer() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr u64 WAIT_LIMIT_NS = 2000000000ull;  // 2 s

// Wait for phase `parity` of `bar`; gives up after WAIT_LIMIT_NS and returns false.
__device__ __forceinline__ bool mbar_wait(u64* bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const u64 t0 = globaltimer();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > WAIT_LIMIT_NS) return false;
    }
}

}  // namespace
}  // namespace dc
