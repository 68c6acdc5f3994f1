// Shared-memory mbarriers and TMA tile loads (cp.async.bulk.tensor) for the
// time-step kernels that stage their rows by TMA. One elected thread of a CTA
// arms a stage's barrier with the byte count it expects and issues the
// copies; every consumer waits on the barrier's phase. Every wait is bounded:
// a wait that gives up returns false, and the kernel then records the failure
// in its error word instead of spinning on.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace lsrtm {
namespace tma {

constexpr unsigned kWaitLimit = 1u << 22;   // mbarrier polls before giving up

__device__ __forceinline__ unsigned su32(const void *p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *b)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase `phase` of barrier b; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned phase)
{
    for (unsigned i = 0; i < kWaitLimit; ++i)
        if (mbar_test(b, phase)) return true;
    return false;
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// its later asynchronous-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Tile loads completing on barrier b; coordinates in elements, innermost first.
__device__ __forceinline__ void load3(void *dst, const CUtensorMap &m, int x, int y, int z, uint64_t *b)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(&m)), "r"(x), "r"(y), "r"(z), "r"(su32(b))
        : "memory");
}
__device__ __forceinline__ void load4(void *dst, const CUtensorMap &m, int x, int y, int z, int q, uint64_t *b)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(&m)), "r"(x), "r"(y), "r"(z), "r"(q), "r"(su32(b))
        : "memory");
}

constexpr unsigned al128(unsigned b) { return (b + 127u) / 128u * 128u; }

}  // namespace tma
}  // namespace lsrtm
