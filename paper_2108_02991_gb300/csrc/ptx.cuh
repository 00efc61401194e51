// Inline-PTX helpers for sm_103a: shared-memory mbarriers, 1-D TMA bulk
// copies (cp.async.bulk) and the SFU reciprocal square root.
#pragma once
#include <cstdint>

#include "kernels.h"

namespace sparkling {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Makes the initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// The wait budget (SM clock cycles) of the context whose status word this is.
__device__ __forceinline__ long long wait_budget(const int *status)
{
    return reinterpret_cast<const volatile DevCtl *>(status)->wait_cycles;
}

// Wait for phase `parity` of the barrier to complete, for at most `budget`
// cycles.  On timeout sets kDevTimeout in *status and returns false.
__device__ __forceinline__ bool mbar_wait_cycles(uint64_t *bar, uint32_t parity, int *status,
                                                 long long budget)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) {
            atomicOr(status, kDevTimeout);
            return false;
        }
    }
    return true;
}

// A wait on data a copy delivers, with the context's budget.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status)
{
    if (mbar_try_wait(bar, parity))
        return true;
    return mbar_wait_cycles(bar, parity, status, wait_budget(status));
}

// After a timeout: wait (with the fixed default budget, whatever the
// context's) for a copy still in flight, so that no bulk copy writes into
// shared memory once the CTA has exited.
__device__ __forceinline__ bool mbar_wait_drain(uint64_t *bar, uint32_t parity, int *status)
{
    return mbar_wait_cycles(bar, parity, status, kWaitCycles);
}

// Arm the barrier for `bytes` of transaction and start a bulk copy of `bytes`
// (multiple of 16, both addresses 16-byte aligned) from global to shared.
__device__ __forceinline__ void bulk_load(void *smem_dst, const void *gmem_src, uint32_t bytes,
                                          uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// MUFU.RSQ: approximate 1/sqrt(x) on the special-function unit, flushing
// subnormal inputs and outputs to zero.
__device__ __forceinline__ float rsqrt_sfu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Paired FP32 arithmetic (two lanes of a 64-bit register, one instruction:
// the f32x2 forms of add, sub, mul and fma of sm_100 and later).
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Error-free transformation of a + b (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Compensated FP32 accumulator (sum + running error term).
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float t, e;
        two_sum(s, x, t, e);
        s = t;
        c += e;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

struct AccD {
    double s = 0.0;
    __device__ __forceinline__ void add(float x) { s += (double)x; }
    __device__ __forceinline__ double value() const { return s; }
};

} // namespace sparkling
