// Binary64 exponentials and quotients on fewer FP64-pipe instructions.
//
// GB300 retires two FP64 FMAs per clock per SM against 128 binary32 FMAs and 64 integer
// operations, so in the FP64 closure one FP64 instruction costs as much pipe time as dozens of
// integer or binary32 ones. These functions keep the binary64 arithmetic that sets the result's
// accuracy and move the rest (range-reduction index, its conversion to binary64, exponent
// scaling, the starting reciprocal) to the integer and binary32 pipes. Accuracy: within 2 ulp of
// the exact result (tested against CUDA's exp and division over the closure's argument ranges);
// arguments outside the fast ranges go to CUDA's own functions.
#pragma once

#include <cuda_runtime.h>

#include "exp_table.h"
#include "fp32.cuh"

namespace hyp {

// Binary64 value of an integer with |n| < 2^31, with integer instructions only.
__device__ __forceinline__ double f64_of_int(int n) {
    if (n == 0) return 0.0;
    const unsigned sign = n < 0 ? 0x80000000u : 0u;
    const unsigned a = n < 0 ? 0u - (unsigned)n : (unsigned)n;
    const int lz = __clz(a);                       // a = 2^(31 - lz) * 1.f
    const unsigned f = (a << lz) << 1;             // the 31 - lz fraction bits, left aligned
    const unsigned hi = sign | ((unsigned)(31 - lz + 1023) << 20) | (f >> 12);
    return __hiloint2double((int)hi, (int)(f << 20));
}

// exp(x) by Tang's table-driven method (ACM TOMS 15(2), 1989): n = nearest integer to
// x 256/ln2 (from a binary32 product: n may be one off the nearest, which only widens the
// reduced range a little), r = x - n ln2/256 in two exact-product FMAs (Cody and Waite's split
// of ln2/256), exp(r) - 1 = r + r^2 (1/2 + r/6 + r^2/24) (Taylor; |r| <= 1.45e-3, the first
// omitted term below 5.3e-17), then 2^(j/256) (1 + p) from the table (j = n mod 256) and 2^m
// (m = floor(n / 256)) added to the exponent field. 7 FP64 instructions. |x| >= 512, NaN and
// infinities take CUDA's exp.
__device__ __forceinline__ double tang_exp(double x) {
    const int hx = __double2hiint(x);
    if (((hx >> 20) & 0x7ff) >= 1023 + 9) return exp(x);
    const float t = fmaf(f32_of(x), EXP_INV_C, 12582912.0f);    // 1.5 * 2^23: round to integer
    const int n = __float_as_int(t) - 0x4B400000;
    const double nd = f64_of_int(n);
    double r = fma(-nd, EXP_C_HI, x);
    r = fma(-nd, EXP_C_LO, r);
    const double r2 = __dmul_rn(r, r);
    double c = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    c = fma(r, c, 0.5);
    const double p = fma(r2, c, r);
    const double tj = EXP_TABLE[n & (EXP_TABLE_N - 1)];
    const double y = fma(tj, p, tj);                              // in [1, 2.003)
    return __hiloint2double(__double2hiint(y) + ((n >> 8) << 20), __double2loint(y));
}

// Approximate binary32 reciprocal (the hardware's rcp.approx, relative error below 2^-22).
__device__ __forceinline__ float rcp_approx_f32(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Reciprocal: binary32 start (|relative error| < 2^-22) refined by two Newton steps in binary64
// (error squared each step: below 2^-88 before the final rounding). |b| outside
// [2^-120, 2^120], zero, NaN and infinities take CUDA's division.
__device__ __forceinline__ bool rcp_fast_range(double b) {
    const int eb = (__double2hiint(b) >> 20) & 0x7ff;
    return eb > 1023 - 120 && eb < 1023 + 120;
}

__device__ __forceinline__ double fast_rcp(double b) {
    if (!rcp_fast_range(b)) return 1.0 / b;
    const double y0 = f64_of(rcp_approx_f32(f32_of(b)));
    const double y1 = fma(y0, fma(-b, y0, 1.0), y0);
    return fma(y1, fma(-b, y1, 1.0), y1);
}

// a / b: the binary64 reciprocal after one Newton step (error < 2^-44), the quotient a y, and one
// correction with its residual a - b q (Markstein's form): within 1 ulp. 5 FP64 instructions.
__device__ __forceinline__ double fast_div(double a, double b) {
    if (!rcp_fast_range(b)) return a / b;
    const double y0 = f64_of(rcp_approx_f32(f32_of(b)));
    const double y1 = fma(y0, fma(-b, y0, 1.0), y0);
    const double q = __dmul_rn(a, y1);
    return fma(fma(-b, q, a), y1, q);
}

}  // namespace hyp
