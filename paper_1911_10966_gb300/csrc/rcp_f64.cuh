// Float64 reciprocal by Newton-Raphson on g(r) = 1/r - x from the hardware approximation (about 23
// bits): each step r <- r + r (1 - x r) doubles the number of correct bits.  Shared by the float64
// residual kernels and the adjoint.
#pragma once

#include <cuda_runtime.h>

namespace esdc {

__device__ __forceinline__ double rcp_approx(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}
__device__ __forceinline__ double rcp_newton1(double x) {     // ~46 bits
    const double r = rcp_approx(x);
    return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ double rcp_newton2(double x) {     // full double precision (within an ulp)
    double r = rcp_newton1(x);
    return fma(r, fma(-x, r, 1.0), r);
}

}  // namespace esdc
