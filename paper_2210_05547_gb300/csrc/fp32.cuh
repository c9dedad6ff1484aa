// Conversions between IEEE-754 binary64 and binary32 with integer operations only.
//
// On GB300 a hardware conversion between double and float issues on the FP64 pipe (two per clock
// per SM, the rate of a DFMA), which is the pipe that bounds the kernels of this library. The
// mixed-precision path (HYP_MIXED) moves work to FP32 and converts its inputs and outputs; doing
// the conversions with integer instructions keeps them off the FP64 pipe.
//
// Both follow the binary formats directly: sign, biased exponent (11 bits, bias 1023 / 8 bits,
// bias 127), fraction (52 / 23 bits).
// * f32_of rounds the fraction to nearest, ties to even (adding one to the packed binary32
//   pattern carries into the exponent, which is the correct result, including overflow to
//   infinity). Magnitudes below the smallest normal binary32 (1.18e-38) become a signed zero;
//   finite magnitudes above the binary32 range become infinity; NaN stays NaN.
// * f64_of is exact for normal binary32 values, zero, infinity and NaN; binary32 subnormals
//   (never produced by f32_of) become a signed zero.
#pragma once

#include <cuda_runtime.h>

namespace hyp {

__device__ __forceinline__ float f32_of(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const unsigned sign = hi & 0x80000000u;
    const int ex = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (ex <= 0) return __uint_as_float(sign);
    if (ex >= 255) {
        const bool nan = ((hi >> 20) & 0x7ffu) == 0x7ffu && (((hi & 0xfffffu) | lo) != 0u);
        return __uint_as_float(sign | 0x7f800000u | (nan ? 0x00400000u : 0u));
    }
    unsigned f = sign | ((unsigned)ex << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;          // the 29 fraction bits dropped
    const unsigned half = 0x10000000u;
    f += (rem > half || (rem == half && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
}

__device__ __forceinline__ double f64_of(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned sign = u & 0x80000000u;
    const unsigned ex = (u >> 23) & 0xffu;
    if (ex == 0u) return __hiloint2double((int)sign, 0);
    const unsigned e64 = ex == 0xffu ? 0x7ffu : ex + (1023u - 127u);
    const unsigned hi = sign | (e64 << 20) | ((u >> 3) & 0xfffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// binary64 -> binary32 by truncating the significand (relative error below 2^-23, towards zero),
// magnitudes below binary32's normal range flushed to a signed zero, finite magnitudes above it
// to infinity. Half the integer instructions of f32_of, for smoothing sums of nonnegative fields
// where that error is immaterial (the mixed path's Gaussian filter of the artificial
// diffusivities); NaN becomes infinity.
__device__ __forceinline__ float f32_trunc(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(u >> 32);
    const int ex = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const unsigned sign = hi & 0x80000000u;
    if (ex <= 0) return __uint_as_float(sign);
    if (ex >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)ex << 23) | ((hi & 0xfffffu) << 3) | ((unsigned)u >> 29));
}

}  // namespace hyp
