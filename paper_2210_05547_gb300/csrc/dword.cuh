// Double-word ("double-float") arithmetic on the binary32 pipe: a value is the unevaluated sum
// h + l of two binary32 numbers with |l| <= ulp(h)/2, about 48 significand bits.
//
// The building blocks are the error-free transforms of Knuth (TwoSum), Dekker (FastTwoSum,
// T. J. Dekker, Numer. Math. 18, 1971) and the FMA form of the product's rounding error; the
// sums and products follow the "sloppy" double-word addition and the double-word product of
// Joldes, Muller and Popescu (ACM TOMS 44(2), 2017), relative error of a few 2^-48 away from
// cancellation. The mixed-precision line operators (HYP_MIXED) use them so that the binary32
// pipe carries the recurrences while the results keep nearly binary64 accuracy: the rounding of
// every binary32 operation is carried in the low word instead of being dropped.
//
// Conversions from and to binary64 use integer instructions (fp32.cuh) except the final sum
// h + l of dw_to_f64, one binary64 addition.
#pragma once

#include <cuda_runtime.h>

#include "fp32.cuh"

namespace hyp {

struct dword {
    float h, l;
};

__device__ __forceinline__ dword two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ dword fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ dword dw_add(dword a, dword b) {
    const dword s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, s.l + (a.l + b.l));
}

__device__ __forceinline__ dword dw_sub(dword a, dword b) {
    return dw_add(a, dword{-b.h, -b.l});
}

__device__ __forceinline__ dword dw_mul(dword a, dword b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}

// binary64 -> double word: h the nearest binary32 (f32_of), l the binary32 nearest to the exact
// remainder x - h, found from the significands with integer operations (x - h needs at most 30
// bits at the scale of x's last place). Remainders below binary32's normal range (|x| < ~1e-31)
// are flushed to zero. |x| beyond binary32's range gives h = +-inf.
__device__ __forceinline__ dword dw_of(double x) {
    const float h = f32_of(x);
    const unsigned long long ux = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((ux >> 52) & 0x7ff);
    const unsigned uh = __float_as_uint(h);
    const int eh = (int)((uh >> 23) & 0xff);
    if (ex == 0 || eh == 0 || eh == 0xff) return {h, 0.0f};
    // significands at the scale 2^(ex - 1075) (x's last place)
    const long long X = (long long)((ux & 0xfffffffffffffULL) | 0x10000000000000ULL);
    const int shift = 29 + (eh - 127) - (ex - 1023);          // 29 or 30 (carry into the exponent)
    const long long H = (long long)((uh & 0x7fffffu) | 0x800000u) << shift;
    long long R = X - H;                                         // |R| <= 2^29
    if (ux >> 63) R = -R;
    const float r = (float)(int)R;                               // rounds to 24 bits
    // r x 2^(ex - 1075): add the scale to r's exponent field when the result stays normal
    if (r == 0.0f) return {h, 0.0f};
    const int er = (int)((__float_as_uint(r) >> 23) & 0xff) + ex - 1075;
    if (er <= 0) return {h, 0.0f};
    return {h, __uint_as_float((__float_as_uint(r) & 0x807fffffu) | ((unsigned)er << 23))};
}

// One step x <- r - c x of a first-order linear recurrence (|c| < 1) with the high and low words
// on two separate dependency chains. The high word takes one product and one sum:
//   c.h x.h = ph + pl exactly (FMA), r.h - ph = sh + sl exactly (two-sum).
// The low word gathers the rounding errors, the low parts and the cross terms:
//   x'.l = (sl - pl) + (r.l - c.l x.h) - c.h x.l.
// The low word's own chain is one FMA, and the rest of its terms come off the high word's chain.
// The pair is left unnormalised: it still represents r - c x to a few 2^-48 of the recurrence's
// scale, and |c| < 1 keeps the low word small. A sequence of steps is thus bound by one product
// and one sum per step, not by a normalised double-word multiply and subtract.
__device__ __forceinline__ dword dw_step(dword x, dword r, dword c) {
    const float ph = __fmul_rn(c.h, x.h);
    const float pl = fmaf(c.h, x.h, -ph);
    const float sh = __fsub_rn(r.h, ph);
    const float bb = __fsub_rn(sh, r.h);
    const float sl = __fadd_rn(__fsub_rn(r.h, __fsub_rn(sh, bb)), __fsub_rn(-ph, bb));
    const float t = __fadd_rn(__fsub_rn(sl, pl), fmaf(-c.l, x.h, r.l));
    return dword{sh, fmaf(-c.h, x.l, t)};
}

__device__ __forceinline__ double dw_to_f64(dword a) { return f64_of(a.h) + f64_of(a.l); }

// the 8-byte forward-sweep slot holding a double word
__device__ __forceinline__ void dw_store(double* p, dword a) {
    *reinterpret_cast<float2*>(p) = make_float2(a.h, a.l);
}
__device__ __forceinline__ dword dw_load(const double* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return {v.x, v.y};
}

}  // namespace hyp
