// tcgen05_common.cuh -- helpers shared by the tensor-core kernels of
// libprism_proj (sm_103a): shared-memory addresses, tcgen05 shared-memory
// matrix descriptors, the MMA commit, warp election and a bounded mbarrier
// wait.  Written from the PTX ISA's descriptions of these instructions.
#pragma once

#include <cstdint>

// 32-bit shared-window address of a pointer into shared memory.
static __device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of tcgen05.mma for a K-major operand without
// swizzle: start address, LBO (bytes between core matrices adjacent in K) and
// SBO (bytes between 8-row groups), all in 16-byte units; descriptor version 1.
static __device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of tcgen05; no swizzle, base offset 0
    return d;
}

// Arrive on the mbarrier once every MMA this thread issued before has completed.
static __device__ __forceinline__ void umma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

// One lane of the (converged) warp.
static __device__ __forceinline__ bool elect_one()
{
    uint32_t pred = 0;
    asm volatile("{\n.reg .pred P;\nelect.sync _|P, 0xffffffff;\nselp.u32 %0, 1, 0, P;\n}\n" : "=r"(pred));
    return pred != 0;
}

// Bounded wait on an mbarrier phase; returns false if the limit ran out.
static __device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit = 1u << 22)
{
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done != 0;
}
