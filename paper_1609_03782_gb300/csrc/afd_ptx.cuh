// Inline-PTX helpers for sm_103a: shared-memory mbarriers with bounded waits
// and TMA (cp.async.bulk.tensor) tile loads.
//
// Every wait in the library is bounded by a %globaltimer deadline.  A wait
// that expires records an error code in the caller-supplied device word
// (first error wins) and returns false; the kernel then leaves its loops, so
// a lost copy or a logic error ends the kernel with a status the host reads
// (afd_sync -> AFD_ETIMEOUT) instead of hanging the GPU.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace afd {

// Wait limit for one mbarrier phase.  A phase normally completes within
// microseconds (one TMA tile or one consumer step).
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

// Error codes written to the device error word.
constexpr int kErrWaitFull = 1;   // a tile load never arrived
constexpr int kErrWaitEmpty = 2;  // consumers never released a ring slot
constexpr int kErrSelfTest = 3;   // afd_selftest_wait: the expected expiry

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Make mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false (and
// records `code` in *err unless an earlier error is there) after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int code,
                                          uint64_t limit_ns = kWaitLimitNs)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity))
                return true;
        if (globaltimer_ns() - t0 > limit_ns) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}

// Bounded wait on an mbarrier given by its 32-bit shared-memory address, with
// a suspend-time hint: a thread whose phase is not complete is suspended in
// the try_wait itself (woken when the phase completes, or after hint_ns)
// instead of spinning on issue slots that the CTA's working warps need.
// Returns false (recording `code` in *err unless an earlier error is there)
// after kWaitLimitNs.
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity,
                                                   uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

#ifndef AFD_WAIT_HINT_NS
#define AFD_WAIT_HINT_NS 100000
#endif
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity, int *err, int code)
{
    constexpr uint32_t kHintNs = AFD_WAIT_HINT_NS;  // per suspension
    if (mbar_try_wait_hint(bar, parity, kHintNs))
        return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait_hint(bar, parity, kHintNs))
            return true;
        if (globaltimer_ns() - t0 > kWaitLimitNs) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive_u32(uint32_t bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 3-D tiled TMA load of the box described by the tensor map into shared
// memory, completing on `bar` (complete_tx).  The x coordinate times the
// element size must be a multiple of 16 bytes; coordinates may be negative
// or past the end (those elements are zero-filled).
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const void *tmap, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Programmatic dependent launch (sm_90+): wait until the grids this one
// depends on have completed and their memory is visible (a no-op when the
// grid was not launched as a programmatic dependent), and let the next grid
// in the stream be scheduled before this one ends.
__device__ __forceinline__ void grid_dep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace afd
