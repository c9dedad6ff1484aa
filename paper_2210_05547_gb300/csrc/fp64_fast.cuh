// Binary64 exponentials, logarithms and quotients on fewer FP64-pipe instructions.
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
#include "log_table.h"
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

// log(x) for x >= 2 by Tang's table-driven method (ACM TOMS 16(4), 1990) in its reciprocal form:
// x = 2^m y with y in [1, 2) and j the top 7 fraction bits of y (integer instructions),
// r = y inv_j - 1 in one FMA (inv_j the binary64 nearest to 1 / c_j, c_j = 1 + (j + 1/2) / 128;
// |r| < 2^-8, rounding error below 2^-61), log1p(r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5 - r^6/6
// (Taylor; the first omitted term below 2e-18), and
// log x = (m LN2_HI + T_j,hi) + (m LN2_LO + T_j,lo + log1p(r)) with T_j = -log(inv_j) from the
// table. No cancellation for x >= 2 (log x >= ln2): within 1 ulp. 11 FP64 instructions. Below
// 2 (where log x may be near zero), at or above 2^1000, and NaN: CUDA's log.
__device__ __forceinline__ double table_log(double x) {
    const int hx = __double2hiint(x);
    const int ex = (hx >> 20) & 0x7ff;
    if (hx < 0x40000000 || ex >= 1023 + 1000) return log(x);
    const int j = (hx >> 13) & (LOG_TABLE_N - 1);
    const double y = __hiloint2double((hx & 0x000fffff) | 0x3ff00000, __double2loint(x));
    const double* t = LOG_TABLE[j];
    const double r = fma(y, t[0], -1.0);
    double c = fma(r, -1.0 / 6.0, 0.2);
    c = fma(r, c, -0.25);
    c = fma(r, c, 1.0 / 3.0);
    c = fma(r, c, -0.5);
    const double p = fma(__dmul_rn(r, r), c, r);
    const double md = f64_of_int(ex - 1023);
    const double hi = fma(md, LOG_LN2_HI, t[1]);
    const double lo = fma(md, LOG_LN2_LO, t[2]) + p;
    return hi + lo;
}

}  // namespace hyp
