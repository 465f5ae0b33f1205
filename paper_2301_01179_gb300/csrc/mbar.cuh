// mbar.cuh -- shared-memory mbarriers (arrive / parity wait) and the global timer used to
// bound every wait on them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace afmm {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// expected arrival count per phase
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// one arrival, release semantics at CTA scope: the caller's earlier shared-memory writes
// are visible to a thread whose wait on this phase succeeds
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// true once the phase of the given parity has completed (acquire semantics); a fresh
// barrier is in phase 0, and a wait on parity 1 refers to the completed phase before it
__device__ __forceinline__ bool mbar_try(uint64_t *mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// as mbar_try, but a thread whose phase is not yet complete is suspended in hardware for up
// to hint_ns nanoseconds (it resumes as soon as the phase completes), so waiting warps take
// no issue slots from the warps they wait for
__device__ __forceinline__ bool mbar_try_sleep(uint64_t *mbar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

}  // namespace afmm
