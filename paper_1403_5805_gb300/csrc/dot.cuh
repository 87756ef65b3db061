// Row-segment dot products shared by the persistent kernels: one 16-byte segment of a matrix row
// (2 FP64, 4 FP32, 8 BF16 or 16 E4M3 values) times the matching iterate values, accumulated in FP64
// (FP64 rows) or FP32 (narrow rows).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstdint>

namespace jac {

template <typename TM>
struct MatTraits;
template <>
struct MatTraits<double> {
  static constexpr int kVec = 2;
  using X = double;
  using Acc = double;
};
template <>
struct MatTraits<float> {
  static constexpr int kVec = 4;
  using X = float;
  using Acc = float;
};
template <>
struct MatTraits<__nv_bfloat16> {
  static constexpr int kVec = 8;
  using X = float;
  using Acc = float;
};
template <>
struct MatTraits<__nv_fp8_e4m3> {
  static constexpr int kVec = 16;
  using X = float;
  using Acc = float;
};


// ---- x loads (L2 only: the iterate is rewritten by other CTAs between sweeps, so L1 may be stale)
__device__ __forceinline__ void load_x(double (&xv)[2], const double* x) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(x));
  xv[0] = v.x;
  xv[1] = v.y;
}
template <int V>
__device__ __forceinline__ void load_x(float (&xv)[V], const float* x) {
#pragma unroll
  for (int q = 0; q < V / 4; ++q) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(x) + q);
    xv[4 * q + 0] = v.x;
    xv[4 * q + 1] = v.y;
    xv[4 * q + 2] = v.z;
    xv[4 * q + 3] = v.w;
  }
}

// ---- one 16-byte segment of a row times the matching x values
__device__ __forceinline__ void seg_dot(double& acc, uint4 m, const double (&xv)[2]) {
  const double m0 = __hiloint2double(static_cast<int>(m.y), static_cast<int>(m.x));
  const double m1 = __hiloint2double(static_cast<int>(m.w), static_cast<int>(m.z));
  acc = fma(m0, xv[0], acc);
  acc = fma(m1, xv[1], acc);
}
__device__ __forceinline__ void seg_dot(float& acc, uint4 m, const float (&xv)[4]) {
  acc = fmaf(__uint_as_float(m.x), xv[0], acc);
  acc = fmaf(__uint_as_float(m.y), xv[1], acc);
  acc = fmaf(__uint_as_float(m.z), xv[2], acc);
  acc = fmaf(__uint_as_float(m.w), xv[3], acc);
}
__device__ __forceinline__ void bf16x2_fma(float& acc, uint32_t w, float x0, float x1) {
  acc = fmaf(__uint_as_float(w << 16), x0, acc);          // element 2q   (low half)
  acc = fmaf(__uint_as_float(w & 0xFFFF0000u), x1, acc);  // element 2q+1 (high half)
}
__device__ __forceinline__ void seg_dot(float& acc, uint4 m, const float (&xv)[8]) {
  bf16x2_fma(acc, m.x, xv[0], xv[1]);
  bf16x2_fma(acc, m.y, xv[2], xv[3]);
  bf16x2_fma(acc, m.z, xv[4], xv[5]);
  bf16x2_fma(acc, m.w, xv[6], xv[7]);
}
__device__ __forceinline__ void e4m3x4_fma(float& acc, uint32_t w, const float* x) {
  const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w & 0xFFFFu), __NV_E4M3);
  const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w >> 16), __NV_E4M3);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
  acc = fmaf(a.x, x[0], acc);
  acc = fmaf(a.y, x[1], acc);
  acc = fmaf(b.x, x[2], acc);
  acc = fmaf(b.y, x[3], acc);
}
__device__ __forceinline__ void seg_dot(float& acc, uint4 m, const float (&xv)[16]) {
  e4m3x4_fma(acc, m.x, xv + 0);
  e4m3x4_fma(acc, m.y, xv + 4);
  e4m3x4_fma(acc, m.z, xv + 8);
  e4m3x4_fma(acc, m.w, xv + 12);
}

// One segment of each of a warp's R rows against the same x values.  FP64: every row's first product,
// then every row's second, so consecutive FMAs are independent (each row's own order is the same as
// seg_dot's).  Narrow rows: seg_dot row by row (their FP32 chains are short-latency).
template <int R>
__device__ __forceinline__ void seg_dot_rows(double (&acc)[R], const uint4 (&m)[R], const double (&xv)[2]) {
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = fma(__hiloint2double(static_cast<int>(m[r].y), static_cast<int>(m[r].x)), xv[0], acc[r]);
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = fma(__hiloint2double(static_cast<int>(m[r].w), static_cast<int>(m[r].z)), xv[1], acc[r]);
}
template <int R, int V>
__device__ __forceinline__ void seg_dot_rows(float (&acc)[R], const uint4 (&m)[R], const float (&xv)[V]) {
#pragma unroll
  for (int r = 0; r < R; ++r) seg_dot(acc[r], m[r], xv);
}

// The segment that straddles the end of a row (columns >= n inside it) may carry row padding that is
// not guaranteed to be zero or even finite when A is read in place.  x is zeroed there, and for FP64
// rows the padding element is skipped, not multiplied (NaN * 0 would poison the sum).  The narrow
// copies are written by this library with zero padding, so their full segment is safe.
template <typename XT, int V>
__device__ __forceinline__ void mask_tail(XT (&xv)[V], int64_t col, int64_t n) {
#pragma unroll
  for (int e = 0; e < V; ++e)
    if (col + e >= n) xv[e] = XT(0);
}
__device__ __forceinline__ void seg_dot_tail(double& acc, uint4 m, const double (&xv)[2], int64_t valid) {
  acc = fma(__hiloint2double(static_cast<int>(m.y), static_cast<int>(m.x)), xv[0], acc);
  if (valid > 1) acc = fma(__hiloint2double(static_cast<int>(m.w), static_cast<int>(m.z)), xv[1], acc);
}
template <int V>
__device__ __forceinline__ void seg_dot_tail(float& acc, uint4 m, const float (&xv)[V], int64_t) {
  seg_dot(acc, m, xv);
}

}  // namespace jac
