// fp_bits.cuh - binary64 <-> binary32 conversions built from the IEEE-754 layouts with integer
// operations only.  On GB300 the F2F conversion instructions run on the narrow FP64 pipe; these
// forms run on the integer pipe instead.
#pragma once

#include <cuda_runtime.h>

namespace {

// FP64 -> FP32 with round-to-nearest-even, built from the IEEE-754 binary64/binary32
// layouts with integer operations only (on GB300 the F2F conversion instruction runs on the
// narrow FP64 pipe).  Outside the normal binary32 range the result is chosen with integer
// selects, so no conversion instruction is issued for any lane: |x| < 2^-126 gives a signed
// zero (binary32 subnormal results are flushed), |x| >= 2^128 and infinities give a signed
// infinity, NaN gives a quiet NaN.  Rounding up at the top of the range carries into the
// exponent and gives infinity, as IEEE rounding does.
__device__ __forceinline__ float d2f_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hi = (unsigned int)(b >> 32);
    const int e = (int)((hi >> 20) & 0x7FFu);
    unsigned int r = ((unsigned int)(e - 896) << 23) | ((unsigned int)(b >> 29) & 0x7FFFFFu);
    const unsigned int rem = (unsigned int)b & 0x1FFFFFFFu;
    r += (rem > 0x10000000u) | ((rem == 0x10000000u) & (r & 1u));
    const bool nan = e == 2047 && (b & 0xFFFFFFFFFFFFFull) != 0ull;
    r = e < 897 ? 0u : r;
    r = e > 1150 ? (nan ? 0x7FC00000u : 0x7F800000u) : r;
    return __uint_as_float(r | (hi & 0x80000000u));
}

// FP32 -> FP64 (exact for normal numbers) from the bit layouts with integer operations only:
// zero and binary32 subnormals give a signed zero (flushed), infinities and NaNs keep their
// class (the low mantissa bits of a NaN stay in the low word).
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned int b = __float_as_uint(x);
    const unsigned int e = (b >> 23) & 0xFFu;
    const unsigned int sg = b & 0x80000000u;
    unsigned int hi = sg | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
    unsigned int lo = (b & 7u) << 29;
    hi = e == 0u ? sg : hi;
    lo = e == 0u ? 0u : lo;
    hi = e == 255u ? (sg | 0x7FF00000u | ((b & 0x7FFFFFu) >> 3)) : hi;
    return __hiloint2double((int)hi, (int)lo);
}

}  // namespace
