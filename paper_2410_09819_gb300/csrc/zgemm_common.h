// Device-side primitives shared by the emulated-update kernels (k_ozaki.cu, k_ozaki64.cu):
// mbarriers with bounded waits, TMA loads, tcgen05 MMA / commit / TMEM loads in inline PTX.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace tc {

__device__ __forceinline__ uint32_t z_smem(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t z_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void z_init(uint64_t *bar, uint32_t c) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(z_smem(bar)), "r"(c) : "memory");
}
__device__ __forceinline__ void z_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(z_smem(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void z_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(z_smem(bar)) : "memory");
}
__device__ __forceinline__ bool z_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(z_smem(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when the phase did not complete within limit_ns or another role of
// the CTA gave up (abort flag in shared memory).
__device__ __forceinline__ bool z_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                       unsigned long long limit_ns) {
    if (z_try(bar, parity)) return true;
    const uint64_t t0 = z_timer();
    for (;;) {
        if (z_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (z_timer() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void z_tma(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            z_smem(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z_smem(bar))
        : "memory");
}
__device__ __forceinline__ void z_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(z_smem(bar))
                 : "memory");
}
__device__ __forceinline__ uint64_t z_desc(uint32_t saddr) {   // K-major, 128-byte swizzle
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}
__device__ __forceinline__ void z_mma(uint32_t d, uint64_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(bdesc), "r"(idesc), "r"(acc));
}
// The 4 MMAs of one 128-byte K block in one asm block: the first K step takes the accumulate
// predicate, the others accumulate; A and B advance by 32 bytes (2 descriptor units) per step.
__device__ __forceinline__ void z_mma4(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %4, 0;\n\tsetp.eq.b32 q, %4, %4;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %5, %6, %3, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %7, %8, %3, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %9, %10, %3, q;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc), "l"(a + 2), "l"(b + 2), "l"(a + 4), "l"(b + 4), "l"(a + 6), "l"(b + 6));
}
// K steps 1..3 of a K block (all accumulate)
__device__ __forceinline__ void z_mma3(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.eq.b32 q, %3, %3;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %4, %5, %3, q;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %6, %7, %3, q;\n\t}\n" ::"r"(d),
        "l"(a + 2), "l"(b + 2), "r"(idesc), "l"(a + 4), "l"(b + 4), "l"(a + 6), "l"(b + 6));
}
__device__ __forceinline__ void z_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 3D tile load (K bytes, rows within a digit plane, plane index): consecutive planes in one copy
__device__ __forceinline__ void z_tma3(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            z_smem(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(z_smem(bar))
        : "memory");
}
// Smallest e with amax <= 2^e (0 for amax <= 0): a tile's digit exponent.
__device__ __forceinline__ int z_digit_exp(double amax) {
    if (!(amax > 0.0)) return 0;
    int ex;
    const double f = frexp(amax, &ex);
    return (f == 0.5) ? ex - 1 : ex;
}

}  // namespace tc
