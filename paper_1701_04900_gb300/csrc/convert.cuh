// FP32 <-> FP64 conversions by the IEEE 754 field layout, on the integer pipes.
//
// GB300 executes FP64 arithmetic, including the F32<->F64 conversion instructions, on a narrow
// pipe: a kernel that converts a residual tile per block (FP64 residual -> FP32 snapshot) and
// an increment per scatter (FP32 -> FP64 reduction operand) spends its time there.  Between
// binary32 and binary64 the conversion is a re-packing of sign, exponent and fraction:
//   binary32: sign(1) exponent(8, bias 127) fraction(23)
//   binary64: sign(1) exponent(11, bias 1023) fraction(52)
// Both functions below give the same bits as the hardware conversion with round-to-nearest-even;
// inputs outside the range they handle (zero and subnormal sources or results, infinities,
// NaN, binary32 overflow) take the hardware conversion.
#pragma once

#include <cstdint>

namespace asyflexa {

// binary32 -> binary64 (exact): the exponent is re-biased by 1023 - 127 = 896 and the 23-bit
// fraction becomes the top of the 52-bit one.
__device__ __forceinline__ double f32_to_f64(float x) {
    const uint32_t f = __float_as_uint(x);
    const uint32_t e = (f >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) {
        if ((f & 0x7fffffffu) == 0u) return __hiloint2double(static_cast<int>(f), 0);  // signed zero
        return static_cast<double>(x);
    }
    const uint32_t hi = (f & 0x80000000u) | ((e + 896u) << 20) | ((f & 0x7fffffu) >> 3);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(f << 29));
}

// binary64 -> binary32, round to nearest, ties to even.  Binary32 normal results have binary64
// exponents 897 .. 1150; the fraction keeps the top 23 of 52 bits, and the 29 dropped bits
// decide the rounding (above half: up; exactly half: up when the kept fraction is odd).  A
// carry out of the fraction raises the exponent, which is the correctly rounded result (up to
// infinity from the largest binade).
__device__ __forceinline__ float f64_to_f32(double d) {
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(d));
    const uint32_t lo = static_cast<uint32_t>(__double2loint(d));
    const uint32_t e = (hi >> 20) & 0x7ffu;
    if (e - 897u > 253u) {  // below 897 wraps around to a large unsigned value
        if ((hi & 0x7fffffffu) == 0u && lo == 0u) return __uint_as_float(hi & 0x80000000u);  // signed zero
        return __double2float_rn(d);
    }
    const uint32_t frac = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1fffffffu;
    const uint32_t up = (rest > 0x10000000u || (rest == 0x10000000u && (frac & 1u))) ? 1u : 0u;
    return __uint_as_float(((hi & 0x80000000u) | ((e - 896u) << 23) | frac) + up);
}

}  // namespace asyflexa
