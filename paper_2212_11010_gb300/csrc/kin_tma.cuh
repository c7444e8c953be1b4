// kin_tma.cuh -- bulk-copy (TMA) and mbarrier helpers in inline PTX for
// sm_100+ / sm_103a, plus division by invariant integers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kin {

// n / d for 0 <= n < 2^31 and 1 <= d < 2^31, by a multiply-high and a shift
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", 1994): with s = ceil(log2 d) and
// mul = floor(2^32 (2^s - d) / d) + 1, q = (mulhi(n, mul) + n) >> s.
struct FastDiv {
    unsigned d, mul, shift;
};

inline FastDiv make_fastdiv(unsigned d)
{
    FastDiv f;
    f.d = d;
    unsigned s = 0;
    while ((1ull << s) < d) ++s;
    f.shift = s;
    f.mul = (unsigned)((((1ull << 32) * ((1ull << s) - d)) / d) + 1);
    return f;
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f)
{
    return (__umulhi(n, f.mul) + n) >> f.shift;
}

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or about 'ns' nanoseconds have passed, instead of polling.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, unsigned parity, unsigned ns)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Wait for phase 'parity' of the barrier for at most 'cycles' SM clocks.
// Between polls the thread sleeps (__nanosleep, growing to 256 ns), so a
// waiting warp issues almost nothing while the bulk copies are in flight.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long cycles)
{
    const long long t0 = clock64();
    unsigned ns = 32;
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > cycles) return false;
        __nanosleep(ns);
        if (ns < 256) ns *= 2;
    }
    return true;
}

// global -> shared bulk copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16 bytes).
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// shared -> global bulk copy tracked by the bulk async-group of this thread.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src_smem, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Wait until the shared-memory sources of this thread's bulk stores have been read.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Make this thread's generic-proxy shared-memory writes visible to the
// async proxy (bulk copies that read shared memory).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}


// ---- 16-byte asynchronous copies through the load/store units ----
// global -> shared without register staging (cp.async, L2 only); completion
// is per thread (cp_wait_all), visibility to the block needs a barrier.
__device__ __forceinline__ void cp16_g2s(void* sdst, const void* gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
// 4- or 8-byte variant (through L1), for sources aligned to their size only
template <int BYTES>
__device__ __forceinline__ void cp_small_g2s(void* sdst, const void* gsrc)
{
    static_assert(BYTES == 4 || BYTES == 8, "cp.async.ca takes 4, 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// all but the N most recent commit groups of this thread have landed
template <int N>
__device__ __forceinline__ void cp_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// all but the most recent commit group of this thread have landed
__device__ __forceinline__ void cp_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

}  // namespace kin
