// Setup kernels: the splitting A = D - L - U of Section 2, kept factored.
//
// The sweep applies T = D^-1 (L + U) without forming it: it streams A itself (or a narrow copy of its
// off-diagonal part) and scales each row by 1/a_ii in the epilogue.  Setup therefore only
//   * reads the diagonal, rejects a_ii == 0 or non-finite (Section 2: the method needs a_ii != 0), and
//     stores d_i = a_ii and rinv_i = 1/a_ii (one correctly rounded reciprocal per row);
//   * copies B and takes ||B||_inf;
//   * for the mixed-precision paths, writes the narrow copy of the off-diagonal part of A (FP32, BF16
//     or E4M3 with an FP32 scale per row) in one pass over A: E4M3 and split-float handles, many right-
//     hand sides, and a copy read out before any solve.  The BF16 / FP32 copies of the other handles are
//     written by the first inner sweep of their first solve (solve.cu), with the same rounding.
// Rounding of the narrow copies: a_ij -> FP32 (round to nearest even), then BF16 round to nearest even;
// for E4M3 the row scale s_i is the smallest power of two with max_{j != i} |a32_ij| <= 448 s_i (s_i = 1 if
// the maximum is 0) and the code is the saturating round-to-nearest-even E4M3 of a32_ij / s_i (exact:
// the product with 1 / s_i).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "device_util.cuh"
#include "f64tof32.cuh"
#include "solver.cuh"
#include "splitfloat.cuh"

namespace jac {
namespace {

constexpr int kPrepThreads = 256;

int prep_blocks(int64_t work, int per_block) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return static_cast<int>(b);
}

__global__ void diag_kernel(const double* __restrict__ A, int64_t lda, int64_t n, double* __restrict__ d,
                            double* __restrict__ rinv, unsigned long long* key) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double a = A[i * lda + i];
    unsigned code = 0;
    if (!isfinite(a))
      code = 3;
    else if (a == 0.0)
      code = 2;
    if (code) atomicMin(key, (static_cast<unsigned long long>(i) << 8) | code);
    d[i] = a;
    rinv[i] = code ? 0.0 : __drcp_rn(a);
  }
}

// b = B, ||b||_inf, and (if cmax_bits) max_i |b_i / a_ii|, the iterate's scale for the split-float residual.
__global__ void rhs_kernel(const double* __restrict__ B, int64_t n, const double* __restrict__ rinv,
                           double* __restrict__ b, unsigned long long* bnorm_bits, unsigned long long* cmax_bits) {
  unsigned long long m = 0, c = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = B[i];
    if (b != B) b[i] = v;
    const unsigned long long bits = abs_bits(v);
    m = bits > m ? bits : m;
    if (cmax_bits) {
      const unsigned long long cb = abs_bits(v * rinv[i]);
      c = cb > c ? cb : c;
    }
  }
  m = warp_max_u64(m);
  c = warp_max_u64(c);
  if ((threadIdx.x & 31) == 0) {
    if (m) atomicMax(bnorm_bits, m);
    if (c) atomicMax(cmax_bits, c);  // c stays 0 without cmax_bits
  }
}

__global__ void pad_zero_kernel(double* M, int64_t n, int64_t ld) {
  const int64_t w = ld - n;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) M[i * ld + n + j] = 0.0;
}

// Four narrow values stored with one instruction (4 x 1, 2 or 4 bytes; the destination is aligned to it
// because ldn is a multiple of 16 and j a multiple of 4).
template <typename TL>
struct alignas(4 * sizeof(TL)) Quad {
  TL v[4];
};

// Elements [j, j + 4) of a row; entries at or past n read as 0 and are never loaded (a borrowed A's row
// padding may hold anything).  Rows start 16-byte aligned (borrowed A: aligned base, even lda).
__device__ __forceinline__ void load_quad(const double* row, int64_t j, int64_t n, double (&a)[4]) {
  if (j + 4 <= n) {
    const double2 v0 = __ldcs(reinterpret_cast<const double2*>(row + j));
    const double2 v1 = __ldcs(reinterpret_cast<const double2*>(row + j + 2));
    a[0] = v0.x;
    a[1] = v0.y;
    a[2] = v1.x;
    a[3] = v1.y;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) a[e] = j + e < n ? row[j + e] : 0.0;
  }
}

// fl32(a_ij) of the quad, 0 on the diagonal and past n.
__device__ __forceinline__ void quad_f32(const double (&a)[4], int64_t j, int64_t n, int64_t i, float (&f)[4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) f[e] = (j + e < n && j + e != i) ? f64_to_f32_rn(a[e]) : 0.0f;
}

template <typename TL>
__device__ __forceinline__ void encode_quad(const float (&f)[4], float s, TL* dst);
template <>
__device__ __forceinline__ void encode_quad<float>(const float (&f)[4], float, float* dst) {
  *reinterpret_cast<float4*>(dst) = make_float4(f[0], f[1], f[2], f[3]);
}
template <>
__device__ __forceinline__ void encode_quad<__nv_bfloat16>(const float (&f)[4], float, __nv_bfloat16* dst) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(f[0], f[1]);  // round to nearest even, pairwise
  const __nv_bfloat162 hi = __floats2bfloat162_rn(f[2], f[3]);
  uint2 w;
  w.x = *reinterpret_cast<const uint32_t*>(&lo);
  w.y = *reinterpret_cast<const uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(dst) = w;
}
template <>
__device__ __forceinline__ void encode_quad<__nv_fp8_e4m3>(const float (&f)[4], float inv_s, __nv_fp8_e4m3* dst) {
  // saturating round-to-nearest-even E4M3 of fl32(a_ij) / s_i; s_i is a power of two, so the quotient is
  // the product with the exact 1 / s_i (the same correctly rounded value as the division)
  const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(__fmul_rn(f[0], inv_s), __fmul_rn(f[1], inv_s)),
                                                           __NV_SATFINITE, __NV_E4M3);
  const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(__fmul_rn(f[2], inv_s), __fmul_rn(f[3], inv_s)),
                                                           __NV_SATFINITE, __NV_E4M3);
  *reinterpret_cast<uint32_t*>(dst) = static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
}

// E4M3 row scale from the bits of m = max_{j != i} |fl32(a_ij)|: the smallest power of two 2^k with
// m <= 448 * 2^k (448 = 1.75 * 2^8: k = e - 8 while m's significand is at most 1.75, else e - 7), k clamped
// to [-126, 127]; 1 for m = 0.  Returns k.
__device__ __forceinline__ int e4m3_scale_exponent(unsigned int mbits) {
  if (mbits >= 0x7F800000u) return 127;
  const int e = static_cast<int>(mbits >> 23);
  if (e == 0) return -126;  // m < 2^-126 <= 448 * 2^-126
  const int k = e - 135 + ((mbits & 0x7FFFFFu) > 0x600000u ? 1 : 0);
  return k < -126 ? -126 : (k > 127 ? 127 : k);
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  T r = 0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) r = sh[w] > r ? sh[w] : r;
  return r;
}

// One CTA per row (grid-stride over rows): narrow copy of the off-diagonal part of row i, padding
// zeroed up to ldn, the row factor of the inner sweep and (if rexp) the row's split-float scale
// exponent.  Each thread converts 4 consecutive elements per step: two 16-byte loads, one store.
template <typename TL, bool kScaled, bool kRexp>
__global__ void __launch_bounds__(kPrepThreads) narrow_kernel(const double* __restrict__ A, int64_t lda, int64_t n,
                                                              TL* __restrict__ Nl, int64_t ldn,
                                                              const double* __restrict__ rinv,
                                                              float* __restrict__ scale, float* __restrict__ rowfac,
                                                              int* __restrict__ rexp) {
  __shared__ unsigned int shs[32];
  const int64_t step = 4 * int64_t(blockDim.x);
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double* row = A + i * lda;
    float s = 1.0f, inv = 1.0f;  // the row scale (a power of two) and its exact reciprocal
    if (kScaled) {
      unsigned int m = 0;  // max_{j != i} |fl32(a_ij)| as bits (non-negative floats order like integers)
      for (int64_t j = 4 * int64_t(threadIdx.x); j < n; j += step) {
        double a[4];
        float f[4];
        load_quad(row, j, n, a);
        quad_f32(a, j, n, i, f);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const unsigned int b = __float_as_uint(f[e]) & 0x7FFFFFFFu;
          if (b <= 0x7F800000u) m = b > m ? b : m;  // NaN does not raise the maximum
        }
      }
      m = block_max(m, shs);
      if (m != 0) {
        const int k = e4m3_scale_exponent(m);
        s = __uint_as_float(static_cast<unsigned int>(k + 127) << 23);
        inv = k == 127 ? 0x1p-127f : __uint_as_float(static_cast<unsigned int>(127 - k) << 23);
      }
    }
    TL* out = Nl + i * ldn;
    uint32_t mb = 0;  // max_j of the high word of |a_ij| (all j)
#pragma unroll 2
    for (int64_t j = 4 * int64_t(threadIdx.x); j < ldn; j += step) {
      double a[4];
      float f[4];
      load_quad(row, j, n, a);
      if constexpr (kRexp) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          mb = max(mb, abs_hi(a[e]));
        }
      }
      quad_f32(a, j, n, i, f);
      encode_quad<TL>(f, inv, out + j);
    }
    if constexpr (kRexp) {
      mb = block_max(mb, shs);
      if (threadIdx.x == 0) rexp[i] = split_exponent_hi(mb);
    }
    if (threadIdx.x == 0) {
      if (kScaled) scale[i] = s;
      rowfac[i] = __fmul_rn(__double2float_rn(rinv[i]), s);
    }
  }
}

__global__ void split_x_kernel(const double* __restrict__ x, int64_t n, const unsigned long long* __restrict__ cmax,
                               float2* __restrict__ xs) {
  const int g = split_exponent(*cmax);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    xs[i] = split_x(x[i], g);
}

// One warp per row: r_i = b_i - sum_j a_ij x_j in FP64, max |r_i| as bits.
__global__ void residual_kernel(const double* __restrict__ A, int64_t lda, int64_t n, const double* __restrict__ b,
                                const double* __restrict__ x, unsigned long long* rmax) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    double acc = 0.0;
    for (int64_t j = lane; j < n; j += 32) acc = fma(A[i * lda + j], x[j], acc);
    acc = warp_sum(acc);
    const unsigned long long bits = abs_bits(b[i] - acc);
    m = bits > m ? bits : m;
  }
  if (lane == 0 && m) atomicMax(rmax, m);
}

}  // namespace

cudaError_t launch_diag(const double* A, int64_t lda, int64_t n, double* d, double* rinv,
                        unsigned long long* key_out, cudaStream_t s) {
  diag_kernel<<<prep_blocks(n, kPrepThreads), kPrepThreads, 0, s>>>(A, lda, n, d, rinv, key_out);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const double* B, int64_t n, const double* rinv, double* b, unsigned long long* bnorm_bits,
                       unsigned long long* cmax_bits, cudaStream_t s) {
  rhs_kernel<<<prep_blocks(n, kPrepThreads), kPrepThreads, 0, s>>>(B, n, rinv, b, bnorm_bits, cmax_bits);
  return cudaGetLastError();
}

cudaError_t launch_split_x(const double* x, int64_t n, const unsigned long long* cmax_bits, float2* xs,
                           cudaStream_t s) {
  split_x_kernel<<<prep_blocks(n, kPrepThreads), kPrepThreads, 0, s>>>(x, n, cmax_bits, xs);
  return cudaGetLastError();
}

cudaError_t launch_pad_zero(double* M, int64_t n, int64_t ld, cudaStream_t s) {
  if (ld <= n) return cudaSuccess;
  pad_zero_kernel<<<prep_blocks(n, 1), 32, 0, s>>>(M, n, ld);
  return cudaGetLastError();
}

template <bool kRexp>
void narrow_launch(Narrow kind, int blocks, const double* A, int64_t lda, int64_t n, void* Nlow, int64_t ldn,
                   const double* rinv, float* scale, float* rowfac, int* rexp, cudaStream_t s) {
  switch (kind) {
    case Narrow::F32:
      narrow_kernel<float, false, kRexp><<<blocks, kPrepThreads, 0, s>>>(A, lda, n, static_cast<float*>(Nlow), ldn,
                                                                         rinv, scale, rowfac, rexp);
      break;
    case Narrow::BF16:
      narrow_kernel<__nv_bfloat16, false, kRexp><<<blocks, kPrepThreads, 0, s>>>(
          A, lda, n, static_cast<__nv_bfloat16*>(Nlow), ldn, rinv, scale, rowfac, rexp);
      break;
    case Narrow::E4M3:
      narrow_kernel<__nv_fp8_e4m3, true, kRexp><<<blocks, kPrepThreads, 0, s>>>(
          A, lda, n, static_cast<__nv_fp8_e4m3*>(Nlow), ldn, rinv, scale, rowfac, rexp);
      break;
  }
}

cudaError_t launch_narrow(Narrow kind, const double* A, int64_t lda, int64_t n, void* Nlow, int64_t ldn,
                          const double* rinv, float* scale, float* rowfac, int* rexp, cudaStream_t s) {
  const int blocks = prep_blocks(n, 1);
  if (rexp)
    narrow_launch<true>(kind, blocks, A, lda, n, Nlow, ldn, rinv, scale, rowfac, rexp, s);
  else
    narrow_launch<false>(kind, blocks, A, lda, n, Nlow, ldn, rinv, scale, rowfac, rexp, s);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* A, int64_t lda, int64_t n, const double* b, const double* x,
                            unsigned long long* rmax_bits, cudaStream_t s) {
  residual_kernel<<<prep_blocks(n, 8), 256, 0, s>>>(A, lda, n, b, x, rmax_bits);
  return cudaGetLastError();
}

}  // namespace jac
