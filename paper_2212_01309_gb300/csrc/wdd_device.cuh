// Device helpers shared by the kernels of libwdd.so: shared-memory addresses, mbarriers with
// bounded waits, 1-D TMA bulk copies, and the analytic probe spectrum.
#pragma once

#include <stdint.h>

namespace wdd {

static __device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

static __device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

static __device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

static __device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

static __device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

static __device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One try_wait with a suspend-time hint: the thread sleeps until the phase completes or about
// `hint_ns` pass, instead of polling (polling threads take issue slots from the warps that do the
// work the barrier waits for).
static __device__ __forceinline__ bool mbar_try_sleep(uint64_t* bar, unsigned parity, unsigned hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase completed, false once about wait_ns have passed.  Each try
// sleeps up to 10 us; the SM cycle counter (converted at the maximum SM clock of 2.07 GHz, so at
// lower clocks the limit is proportionally longer) is checked between tries.
static __device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, uint64_t wait_ns) {
    if (mbar_try(bar, parity)) return true;
    const long long limit = (long long)(wait_ns * 2.07);
    const long long t0 = clock64();
    for (unsigned i = 1; i != 0; ++i) {   // also capped at 2^32 tries
        if (mbar_try_sleep(bar, parity, 10000u)) return true;
        if (clock64() - t0 > limit) return false;
    }
    return false;
}

static __device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

static __device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Probe spectrum at a detector point k (pixels) given its squared radius k2 (already rounded):
// A(k) exp(-i coef k2) with A the hard-edged aperture |k|^2 <= R^2 (Algorithm 1 initialisation).
static __device__ __forceinline__ double2 probe_at(double k2, double R2, double coef) {
    if (!(k2 <= R2)) return make_double2(0.0, 0.0);
    if (coef == 0.0) return make_double2(1.0, 0.0);
    double s, c;
    sincos(__dmul_rn(coef, k2), &s, &c);
    return make_double2(c, -s);
}

}  // namespace wdd
