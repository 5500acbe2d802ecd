// tma.cuh -- bulk asynchronous copies (TMA, cp.async.bulk) from global to
// shared memory, completed on an mbarrier, with bounded waits.
//
// Every wait here gives up after a limit of %globaltimer nanoseconds (kWaitNs,
// 2 s, unless the launch carries its own): it then sets a bit in the caller's
// device error word and reports failure, so a kernel never spins forever.  The
// host maps a set word to CUBIC_ERR_TIMEOUT.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cubic {

constexpr unsigned kDevErrTimeout = 1u;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make the initialised barrier visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *smem_dst, const void *gsrc, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Hint: start bringing `bytes` (multiple of 16, 16-byte aligned address) of global memory
// into L2.  Nothing waits for it and it changes no value a later load sees.
__device__ __forceinline__ void bulk_prefetch_l2(const void *gsrc, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}

// Programmatic dependent launch.  pdl_trigger: this CTA lets the next kernel in the
// stream start launching (it runs only its constant prologue before pdl_wait).
// pdl_wait: block until every grid this one depends on has completed and its memory
// is visible.  Both are no-ops for a kernel launched without the PDL attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return done != 0;
}

// Wait for phase `phase` of `bar` to complete, at most limit_ns (0: kWaitNs).  On
// timeout sets kDevErrTimeout in *err and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase, unsigned *err,
                                                  unsigned long long limit_ns = 0)
{
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long lim = limit_ns ? limit_ns : kWaitNs;
    const unsigned long long t0 = global_timer_ns();
    while (!mbar_try_wait(bar, phase)) {
        if (global_timer_ns() - t0 > lim) {
            if (err) atomicOr(err, kDevErrTimeout);
            return false;
        }
    }
    return true;
}

}  // namespace cubic
