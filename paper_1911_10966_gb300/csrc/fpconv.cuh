// float32 <-> float64 conversions on the integer pipe.  On GB300 the float64 pipe issues two
// operations per clock per SM, and the hardware conversions occupy it; the update kernels of the
// mixed-precision form convert every element and would otherwise be bound by those conversions.
// Both follow the IEEE 754 binary32/binary64 encodings; values outside the ranges handled here
// (zeros, subnormals, infinities, NaNs, float results that are subnormal or overflow) take the
// hardware conversion, so every input converts exactly as (double)f and (float)x do.
#pragma once

#include <cuda_runtime.h>

namespace esdc {

// The hardware conversions of the rare cases, kept out of line: inline, the compiler would evaluate
// them unconditionally beside the integer path and select, putting one float64-pipe conversion on
// every element again.
static __device__ __noinline__ double f2d_hw(float f) { return (double)f; }
static __device__ __noinline__ float d2f_hw(double x) { return (float)x; }

// exact float -> double: rebias the exponent (127 -> 1023) and widen the 23-bit significand
__device__ __forceinline__ double f2d_int(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return f2d_hw(f);
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xFFFFFu);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// double -> float, round to nearest even: keep 23 of the 52 significand bits, round on the 29
// dropped ones (ties to the even kept value); a carry out of the significand increments the
// exponent, and one out of the largest finite exponent gives infinity, as the standard requires
__device__ __forceinline__ float d2f_int(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7FFu;
    if (e < 897u || e > 1150u) return d2f_hw(x);         // float zero/subnormal/overflow/inf/nan range
    const unsigned kept = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // 23 bits
    const unsigned rest = lo & 0x1FFFFFFFu;                       // 29 dropped bits
    const unsigned half = 0x10000000u;
    const unsigned up = (rest > half || (rest == half && (kept & 1u))) ? 1u : 0u;
    const unsigned bits = ((hi & 0x80000000u) | ((e - 896u) << 23)) + kept + up;
    return __uint_as_float(bits);
}

}  // namespace esdc
