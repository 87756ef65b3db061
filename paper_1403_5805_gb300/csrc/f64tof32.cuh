// FP64 -> FP32 rounding to nearest even on the integer units.
//
// On GB300 the hardware conversion of a double to a float is issued to the FP64 pipe, at the FP64 FMA rate
// (about 2 per clock per SM, measured 595 G/s against 500 G/s of DFMA), so a pass that narrows every entry
// of an FP64 matrix is bound by that pipe rather than by HBM.  For the normal FP32 range this function
// builds the result from the bits with a few integer instructions; zeros, subnormal results, overflow,
// infinities and NaN take the hardware conversion, so the result equals __double2float_rn for every input.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace jac {

__device__ __forceinline__ float f64_to_f32_rn(double a) {
  const uint32_t hi = static_cast<uint32_t>(__double2hiint(a)), lo = static_cast<uint32_t>(__double2loint(a));
  const uint32_t e = (hi >> 20) & 0x7FFu;
  if (e - 897u > 253u) return __double2float_rn(a);  // FP32 exponent outside 1 .. 254
  // bits 31..23: the low 9 bits of the FP64 exponent, 22..0: the top 23 fraction bits; subtracting
  // 384 << 23 re-biases the exponent (1023 -> 127) modulo 512, which is exact for results in range
  uint32_t t = __funnelshift_l(lo, hi, 3) - 0xC0000000u;
  t = (t & 0x7FFFFFFFu) | (hi & 0x80000000u);
  const uint32_t rb = lo & 0x1FFFFFFFu;  // the 29 dropped fraction bits
  t += (rb > 0x10000000u || (rb == 0x10000000u && (t & 1u))) ? 1u : 0u;  // a carry rounds into the exponent
  return __uint_as_float(t);
}

}  // namespace jac
