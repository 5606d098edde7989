// async.cuh -- shared-memory mbarriers and TMA tensor copies (PTX), used by
// the tensor-core closure tile and the TMA-fed 3-D curl stencils.  Every
// wait is bounded (after max_iter polls, or after a wall-clock limit) and
// returns false when it gives up, so that a kernel can record an error and
// end instead of hanging.
#pragma once

#include <cstdint>

namespace fp {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait on the mbarrier phase; returns false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity, uint32_t max_iter)
{
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(m)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait on the mbarrier phase with the thread suspended in the barrier between
// polls (suspend-time hint 0.5 ms: a waiting warp takes no issue slots and
// wakes when the phase completes); gives up after limit_ns of wall-clock time
__device__ __forceinline__ bool mbar_wait_timed(uint64_t *m, uint32_t parity, uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (bool first = true;; first = false) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(m)), "r"(parity), "r"(500000u)
            : "memory");
        if (ok) return true;
        const uint64_t t = globaltimer_ns();
        if (first)
            t0 = t;
        else if (t - t0 > limit_ns)
            return false;
    }
}

// arrive on the barrier (one of its `count` arrivals) and add `bytes` to the
// transaction count the current phase waits for
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *m, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}

// one of the barrier's `count` arrivals (release: this thread's earlier shared-memory reads are done)
__device__ __forceinline__ void mbar_arrive(uint64_t *m)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(m)) : "memory");
}

// contiguous bulk copy global -> this CTA's shared memory, completion counted
// in bytes on mbarrier m; both addresses 16-byte aligned, bytes a multiple of
// 16.  evict_first: the source is streamed once (an L2 eviction-priority hint).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *m, bool evict_first)
{
    if (evict_first) {
        uint64_t pol;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
            ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(m)), "l"(pol)
            : "memory");
    } else {
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(m))
                     : "memory");
    }
}

// tiled 2-D tensor load global -> shared (as tma_load_3d, one dimension fewer)
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, uint64_t *m, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(tmap), "r"(x), "r"(y), "r"(smem_addr(m))
        : "memory");
}

// tiled 3-D tensor load global -> shared (box given by the tensor map),
// completion counted in bytes on mbarrier m; coordinates are element
// indices (x innermost), out-of-range elements are filled with zero
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, uint64_t *m, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_addr(m))
        : "memory");
}

}  // namespace fp
