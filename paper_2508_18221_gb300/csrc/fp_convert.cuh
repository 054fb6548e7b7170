// FP64 <-> FP32 conversions with integer instructions and selects, for the FP32 algebra of
// the mixed-precision modes.
//
// GB300 executes the hardware conversions (F2F) on its FP64 pipe, which issues about 1/64
// of the integer rate; kernels that convert every input and output (the FP32 right-hand
// side, the FP32 fluxes, the tensor-core line tiles) were bound by it.  Narrowing keeps the
// leading 23 bits of the FP64 mantissa, rounded to nearest even on the 29 dropped bits (a
// carry steps the exponent, up to Inf); widening appends 29 zero bits.  Both give the
// hardware's bits except below FP32's normal range (|x| < 2^-126 ~ 1.2e-38), which becomes
// a signed zero instead of an FP32 subnormal -- irrelevant at FP32 precision and keeping
// the code free of branches, which would stop the compiler from batching the loads that
// feed the conversions.  Inf and NaN stay Inf and NaN.
#pragma once

#include <stdint.h>

namespace gk {

__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t s = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);      // leading 23 mantissa bits
    const uint32_t rest = lo & 0x1FFFFFFFu, half = 0x10000000u;  // the 29 dropped bits
    const uint32_t up = (rest > half || (rest == half && (m & 1u))) ? 1u : 0u;
    const uint32_t normal = (s | ((uint32_t)e << 23) | m) + up;
    const bool nan = e == 2047 - 1023 + 127 && ((hi & 0xFFFFFu) | lo) != 0u;
    const uint32_t big = s | 0x7F800000u | (nan ? 0x00400000u : 0u);
    return __uint_as_float(e >= 255 ? big : (e >= 1 ? normal : s));
}

__device__ __forceinline__ double f2d(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t s = u & 0x80000000u, ef = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    const uint32_t eh = ef == 255u ? 0x7FF00000u : ((ef + 896u) << 20);
    return __hiloint2double((int)(ef == 0u ? s : (s | eh | (m >> 3))), (int)(ef == 0u ? 0u : (m << 29)));
}

// FP64 -> the algebra type R (identity for FP64)
template <class R> __device__ __forceinline__ R narrow(double x);
template <> __device__ __forceinline__ double narrow<double>(double x) { return x; }
template <> __device__ __forceinline__ float narrow<float>(double x) { return d2f_rn(x); }

// the algebra type -> FP64 (identity for FP64)
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float x) { return f2d(x); }

}  // namespace gk
