// cp_async.cuh -- per-thread asynchronous global -> shared copies (cp.async,
// Ampere-style: each thread waits for its own groups and reads back only what
// it copied, so no barrier is involved) and an L1 prefetch.
#pragma once

#include <cstdint>

namespace fp {

// 16 bytes, both addresses 16-byte aligned; bypasses L1
__device__ __forceinline__ void cpa16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
// 4 bytes, both addresses 4-byte aligned
__device__ __forceinline__ void cpa4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// every copy group of this thread has landed
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

}  // namespace fp
