// Inline-PTX building blocks of the tcgen05 kernels (sm_103a): mbarriers with
// bounded waits, TMA tile loads, shared-memory matrix descriptors, TF32 and
// FP16 MMAs with tensor-memory accumulators, and tensor-memory loads.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace g4ptx {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait.  Returns false when the budget ran out (the flag is then set)
// or another role of the block has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget,
                                          volatile int* abort_flag) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Bounded wait for work this block started itself (always completes).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity) && clock64() - t0 < budget) {
    }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_k128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// Instruction descriptor of kind::f16: D = F32, A = B = F16, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// Operand scaling of the FP16 hi/lo splits.  Every operand of one GEMM is
// multiplied by the same power of two 2^s, chosen from the largest magnitude
// among them (maxbits: its FP32 bit pattern, non-negative) so that the scaled
// values stay below 2^14: the hi parts keep a 4x margin to the FP16 maximum
// (65504) and the lo parts (2^-11 below their hi part) stay normal down to
// magnitudes 2^-17 below the largest.  The product of two operands then
// carries 2^(2s), removed exactly from the FP32 result.  s is clamped to
// [-60, 60] so that 2^(+-2s) is a normal FP32 number.
__device__ __forceinline__ int f16_shift(uint32_t maxbits) {
    const int e = (int)((maxbits >> 23) & 0xFFu);
    if (e == 0 || e == 0xFF) return 0;  // zero, subnormal, infinite or NaN largest value
    // max < 2^(e - 126): scaled by 2^(140 - e) it stays below 2^14
    const int s = 140 - e;
    return s < -60 ? -60 : (s > 60 ? 60 : s);
}

// 2^e for e in [-126, 127], exactly.
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Eight consecutive 32-bit columns of this thread's lane into v[0..7].
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// FP32 -> FP64 widening on the integer pipes.  GB300's FP64 pipe is narrow:
// an epilogue that widens every accumulator value with cvt.f64.f32 is bound by
// it, so the epilogues widen half of their values here and half in hardware.
// Normal numbers and zero are converted exactly and branch-free (rebias the
// exponent by 1023 - 127 = 896, 0x380 in the high word); infinity and NaN go
// through the hardware conversion; FP32 subnormals (|x| < 2^-126) become a
// signed zero, an absolute error below 1.2e-38.  The result is negated when
// neg is set (an exact sign flip).
__device__ __forceinline__ double f32_to_f64(float f, bool neg = false) {
    const uint32_t u = __float_as_uint(f) ^ (neg ? 0x80000000u : 0u);
    const uint32_t e = u & 0x7F800000u;
    if (e == 0x7F800000u) return (double)__uint_as_float(u);
    const uint32_t s = u & 0x80000000u;
    const uint32_t hi = e ? (s | (((u & 0x7FFFFFFFu) >> 3) + 0x38000000u)) : s;
    const uint32_t lo = e ? (u << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// FP64 -> FP32 narrowing, round to nearest even, on the integer pipes for
// results in the FP32 normal range (exponent field of the double in
// [897, 1150]); anything else (zero, tiny or huge values, infinity, NaN) goes
// through the hardware conversion.  Kernels that narrow many values use it for
// half of them, spreading the work over the FP64 and integer pipes.
__device__ __forceinline__ float f64_to_f32(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const uint32_t e = (hi >> 20) & 0x7FFu;
    if (e < 897u || e > 1150u) return __double2float_rn(d);
    // sign | rebiased exponent and the top 20 mantissa bits | next 3 bits
    uint32_t bits = (hi & 0x80000000u) | ((((hi & 0x7FFFFFFFu) - 0x38000000u) << 3) | (lo >> 29));
    // round to nearest, ties to even (a carry may reach the exponent, or infinity)
    const uint32_t rest = lo & 0x1FFFFFFFu;
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u))) ? 1u : 0u;
    return __uint_as_float(bits);
}

// Compensated FP32 pairs (an accumulator entry (hi, lo) stands for hi + lo):
// add b to the pair with Knuth's two-sum (the exact rounding error of hi + b)
// and renormalise with a fast two-sum, so that |lo| <= ulp(hi)/2.  The
// intrinsics keep the compiler from contracting or reassociating the steps.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float b) {
    const float s = __fadd_rn(hi, b);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    const float l = __fadd_rn(lo, e);
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
}

// An FP64 value into a pair: its FP32 rounding and the FP32 rounding of the
// rest (exact to about 2^-48 relative).
__device__ __forceinline__ void pair_add(float& hi, float& lo, double x) {
    const float b = __double2float_rn(x);
    const float r = __double2float_rn(x - (double)b);
    pair_add(hi, lo, b);
    pair_add(hi, lo, r);
}

// A complex accumulator entry of pairs: (hi.re, hi.im, lo.re, lo.im), 16 bytes
// like one complex128.
__device__ __forceinline__ void pair_add_c(float4* p, float re, float im) {
    float4 a = *p;
    pair_add(a.x, a.z, re);
    pair_add(a.y, a.w, im);
    *p = a;
}

}  // namespace g4ptx
