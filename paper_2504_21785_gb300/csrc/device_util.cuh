// Device helpers shared by the reconstruction kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

namespace fgr {

// Box window of a Gaussian centred at c on one grid axis (see fgr.h):
//   m_lo = ceil(((c - rs) - lo) / h),  m_hi = floor(((c + rs) - lo) / h),
// clipped to [0, n) (empty when m_lo > m_hi).  Evaluated with explicit
// round-to-nearest operations so that no contraction changes the decision.
__device__ __forceinline__ void window_bounds(double c, double rs, double lo, double h, int64_t n,
                                              int64_t *mlo, int64_t *mhi) {
    double a = __ddiv_rn(__dsub_rn(__dsub_rn(c, rs), lo), h);
    double b = __ddiv_rn(__dsub_rn(__dadd_rn(c, rs), lo), h);
    a = ceil(a);
    b = floor(b);
    a = fmin(fmax(a, 0.0), (double)n);
    b = fmin(fmax(b, -1.0), (double)(n - 1));
    *mlo = (int64_t)a;
    *mhi = (int64_t)b;
}

// q = x / step with floor(q) equal to floor of the correctly rounded quotient:
// x * (1/step) differs from it by a few ulps, so it decides the floor unless it
// lies within 1e-9 (relative) of an integer, where the division is done.
__device__ __forceinline__ double quotient_for_floor(double x, double step, double inv_step) {
    const double r = x * inv_step;
    const double n = rint(r);
    if (fabs(r - n) <= 1e-9 * fmax(1.0, fabs(r))) return __ddiv_rn(x, step);
    return r;
}

// floor(fl(x / step)) as an int, mostly without FP64 arithmetic: the FP32
// product (float)x * (float)inv_step has a relative error below 2e-7, so when
// it lies more than 1e-6 (relative) away from an integer its floor is the
// floor of the exact quotient; otherwise (and for |x/step| >= 1e6) the FP64
// path above decides.
__device__ __forceinline__ int floor_div_int(double x, double step, double inv_step) {
    const float rf = (float)x * (float)inv_step;
    const float fl = floorf(rf);
    const float fr = rf - fl;
    const float tol = 1e-6f * fmaxf(1.f, fabsf(rf));
    if (fabsf(rf) < 1e6f && fr > tol && fr < 1.f - tol) return (int)fl;
    const double r = floor(quotient_for_floor(x, step, inv_step));
    return (int)fmin(fmax(r, -1e9), 1e9);
}

// Grid coordinate x_m = lo + m*h without contraction.
__device__ __forceinline__ double grid_x(double lo, double h, int64_t m) {
    return __dadd_rn(lo, __dmul_rn((double)m, h));
}

// Round to nearest integer for |x| < 2^22 with two FP32 additions on the FMA pipe.
__device__ __forceinline__ float rint_fast(float x) {
    const float magic = 12582912.0f;  // 1.5 * 2^23
    return __fsub_rn(__fadd_rn(x, magic), magic);
}

// 2^x on the special-function unit (relative error about 2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void atomic_add_c(float2 *p, float re, float im) {
    atomicAdd(p, make_float2(re, im));
}

__device__ __forceinline__ void atomic_add_c(double2 *p, double re, double im) {
    atomicAdd(&p->x, re);
    atomicAdd(&p->y, im);
}

}  // namespace fgr
