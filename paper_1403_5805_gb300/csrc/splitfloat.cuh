// Split-float arithmetic: FP64-accurate dot products on GB300's FP32 units, shared by the residual
// passes of the single-system, many-right-hand-side, batched and serving kernels.
//
// GB300 issues about 2 FP64 FMA per clock per SM, so an FP64 pass over A is bound by FP64 arithmetic
// (8 bytes per FMA, ~4.8 TB/s).  The residual only needs FP64-level accuracy, not FP64 instructions:
// each a_ij (scaled by 2^-e_i, e_i the exponent of the row maximum, so |a| < 1) is split with integer
// operations into hi = its top 24 significant bits and lo = the next 23, x_j into two rounded FP32
// words, and the products are accumulated as float-float: the rounding error of hi*hi is recovered
// exactly with an FMA, the two cross products are added to it, and a two-sum (Knuth) keeps the running
// sum as an unevaluated pair.  The representation error is below 2^-46 per element; the lane sums
// leave FP32 as FP64 values scaled back by 2^e_i.  The iterate's two FP32 words (of x scaled by 2^-g, g
// the exponent of max_i |b_i / a_ii|, so any scale of B stays inside FP32's range) are written once per
// outer step by the code that forms the iterate, so a residual pass issues no FP64 instruction per
// element of A.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace jac {

struct FF {
  float hi, lo;
};

__device__ __forceinline__ void split_scaled(double a, int sh, float& hi, float& lo) {
  // branch-free: out-of-range parts (below FP32's normal range relative to the row maximum) become 0
  const uint32_t hw = static_cast<uint32_t>(__double2hiint(a)), lw = static_cast<uint32_t>(__double2loint(a));
  const int E = static_cast<int>((hw >> 20) & 0x7FFu) - sh;  // biased exponent of a * 2^-sh
  const uint32_t sign = hw & 0x80000000u;
  const int fe = E - 896;                                     // FP32 exponent field of hi
  const float h = __uint_as_float(sign | (static_cast<uint32_t>(fe) << 23) | (__funnelshift_l(lw, hw, 3) & 0x7FFFFFu));
  hi = fe > 0 ? h : 0.0f;
  const uint32_t m23 = (lw >> 6) & 0x7FFFFFu;                 // mantissa bits 28..6: the next 23 bits
  const float ml = __fsub_rn(__uint_as_float(0x4B000000u | m23), 8388608.0f);  // m23, exactly
  const float p2 = __uint_as_float(static_cast<uint32_t>(max(E - 942, 0)) << 23);  // 2^(e - 46), or 0
  lo = __uint_as_float(__float_as_uint(__fmul_rn(ml, p2)) | sign);
}

// Renormalise the pair (fast two-sum, |lo| <= |hi|): keeps |lo| <= ulp(hi) / 2, so that the FP32
// additions into lo lose at most 2^-48 |sum| each however many terms a pair accumulates.  Called every
// few products (between calls lo grows by at most about one ulp(hi) per product).
__device__ __forceinline__ void ff_renorm(FF& s) {
  const float z = __fadd_rn(s.hi, s.lo);
  s.lo = __fsub_rn(s.lo, __fsub_rn(z, s.hi));
  s.hi = z;
}

__device__ __forceinline__ void ff_fma(FF& s, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  const float e = __fmaf_rn(ah, xh, -p);  // exact error of the rounded product
  const float t = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
  const float u = __fadd_rn(s.hi, p);  // two-sum of s.hi and p
  const float v = __fsub_rn(u, s.hi);
  const float w = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(u, v)), __fsub_rn(p, v));
  s.hi = u;
  s.lo = __fadd_rn(s.lo, __fadd_rn(w, t));
}

// 2^e as a double for -1022 <= e <= 1023 (exact; built from the exponent field).
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double(static_cast<long long>(1023 + e) << 52); }

// Exponent used to scale a row of A or a vector for the split: e with max |v| < 2^e, clamped so that
// 2^e and 2^-e are normal doubles; 0 for a zero or non-finite maximum.  bits: IEEE bits of max |v|.
__device__ __forceinline__ int split_exponent(unsigned long long bits) {
  const int be = static_cast<int>((bits >> 52) & 0x7FFu);
  if (be == 0x7FF || bits == 0) return 0;
  const int e = be == 0 ? -1000 : be - 1022;  // |v| < 2^(be - 1022) for normal v
  return e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
}

// The same exponent from the maximum of the high 32 bits of |v| (sign cleared): the exponent field and
// the zero / subnormal / non-finite cases sit there, so a 32-bit running maximum suffices.
__device__ __forceinline__ uint32_t abs_hi(double v) {
  return static_cast<uint32_t>(__double2hiint(v)) & 0x7FFFFFFFu;
}
__device__ __forceinline__ int split_exponent_hi(uint32_t hi_bits) {
  return split_exponent(static_cast<unsigned long long>(hi_bits) << 32);
}

// x * 2^-g as an unevaluated pair of FP32 words: hi = fl32(x 2^-g), lo = fl32(x 2^-g - hi).
__device__ __forceinline__ float2 split_x(double x, int g) {
  const double v = x * pow2(-g);
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - static_cast<double>(hi)));
}

}  // namespace jac
