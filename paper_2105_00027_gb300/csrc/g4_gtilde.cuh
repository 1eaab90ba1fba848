// One entry of a measurement's sign-weighted Green's function, in FP32, as the
// mixed path stores it (device code shared by the G build, the largest-|G~|
// pass and the kernels that form the tensor-core operands straight from M):
//
//   G~(K1, K2) = r_s [G0(K1) delta(K1, K2) - G0(K1) M(K1, K2) G0(K2)]
//
// (G = G0 delta - G0 M G0 is how the walker's M gives G, Sec. 2), where the
// factor r_s = sqrt(|s|) for a measurement of sign s >= 0 and i sqrt(|s|) for
// s < 0, so that the product of two entries of the same measurement carries
// its sign s.  The products run left to right: (G0(K1) M) G0(K2).
#pragma once

#include <cuda_runtime.h>

#include "g4_ptx.cuh"

namespace g4gt {

// The sign factor of a measurement: magnitude sqrt(|s|) and whether it is i
// times that (s < 0).
struct SignFactor {
    float rs;
    bool neg;
};

__host__ __device__ inline SignFactor sign_factor(double sign) {
    SignFactor f;
    f.rs = (float)sqrt(fabs(sign));
    f.neg = sign < 0.0;
    return f;
}

// gi = G0(K1), m = M(K1, K2), gj = G0(K2), diag = (K1 == K2).  Every operation
// is an explicit round-to-nearest intrinsic (each complex product component is
// one multiply and one fused multiply-add), so that every kernel that forms G~
// gets the same bits whatever the compiler would contract around it.
__device__ __forceinline__ float2 cmul_fixed(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}

__device__ __forceinline__ float2 g_tilde(float2 gi, float2 m, float2 gj, bool diag, SignFactor f) {
    const float2 p = cmul_fixed(cmul_fixed(gi, m), gj);
    float2 v = make_float2(-p.x, -p.y);
    if (diag) {
        v.x = __fadd_rn(v.x, gi.x);
        v.y = __fadd_rn(v.y, gi.y);
    }
    v.x = __fmul_rn(v.x, f.rs);
    v.y = __fmul_rn(v.y, f.rs);
    if (f.neg) v = make_float2(-v.y, v.x);
    return v;
}

// An entry of M as complex64: complex64 as stored; complex128 rounded to
// nearest (the real part by the hardware conversion, the imaginary part on the
// integer pipes, to spread the narrowing over both).
__device__ __forceinline__ float2 to_c64(float2 m) { return m; }
__device__ __forceinline__ float2 to_c64(double2 m) {
    return make_float2((float)m.x, g4ptx::f64_to_f32(m.y));
}

}  // namespace g4gt
