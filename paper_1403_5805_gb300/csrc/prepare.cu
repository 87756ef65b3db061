// Setup kernels: the splitting A = D - L - U of Section 2, kept factored.
//
// The sweep applies T = D^-1 (L + U) without forming it: it streams A itself (or a narrow copy of its
// off-diagonal part) and scales each row by 1/a_ii in the epilogue.  Setup therefore only
//   * reads the diagonal, rejects a_ii == 0 or non-finite (Section 2: the method needs a_ii != 0), and
//     stores d_i = a_ii and rinv_i = 1/a_ii (one correctly rounded reciprocal per row);
//   * copies B and takes ||B||_inf;
//   * for the mixed-precision paths, writes the narrow copy of the off-diagonal part of A (FP32, BF16
//     or E4M3 with an FP32 scale per row) in one pass over A.
// Rounding of the narrow copies: a_ij -> FP32 (round to nearest even), then BF16 round to nearest even;
// for E4M3 the row scale s_i = max_{j != i} |a32_ij| / 448 (FP32 division, s_i = 1 if that is 0) and
// the code is the saturating round-to-nearest-even E4M3 of a32_ij / s_i (FP32 division).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "device_util.cuh"
#include "solver.cuh"

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

__global__ void rhs_kernel(const double* __restrict__ B, int64_t n, double* __restrict__ b,
                           unsigned long long* bnorm_bits) {
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = B[i];
    if (b != B) b[i] = v;
    const unsigned long long bits = abs_bits(v);
    m = bits > m ? bits : m;
  }
  m = warp_max_u64(m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(bnorm_bits, m);
}

__global__ void pad_zero_kernel(double* M, int64_t n, int64_t ld) {
  const int64_t w = ld - n;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < w; j += blockDim.x) M[i * ld + n + j] = 0.0;
}

__device__ __forceinline__ float block_max_abs(float v, float* sh) {
  // non-negative floats: the IEEE encodings order like unsigned integers
  unsigned int u = __float_as_uint(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned int w = __shfl_xor_sync(0xffffffffu, u, o);
    u = w > u ? w : u;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = __uint_as_float(u);
  __syncthreads();
  unsigned int r = 0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
    const unsigned int x = __float_as_uint(sh[w]);
    r = x > r ? x : r;
  }
  return __uint_as_float(r);
}

template <typename TL>
__device__ __forceinline__ TL narrow_encode(float a32, float s);
template <>
__device__ __forceinline__ float narrow_encode<float>(float a32, float) {
  return a32;
}
template <>
__device__ __forceinline__ __nv_bfloat16 narrow_encode<__nv_bfloat16>(float a32, float) {
  return __float2bfloat16_rn(a32);
}
template <>
__device__ __forceinline__ __nv_fp8_e4m3 narrow_encode<__nv_fp8_e4m3>(float a32, float s) {
  __nv_fp8_e4m3 q;
  q.__x = __nv_cvt_float_to_fp8(__fdiv_rn(a32, s), __NV_SATFINITE, __NV_E4M3);
  return q;
}

// One CTA per row (grid-stride): narrow copy of the off-diagonal part of row i, padding zeroed up to
// ldn, and the row factor of the inner sweep.
__device__ __forceinline__ unsigned long long block_max_bits(unsigned long long v, unsigned long long* sh) {
  v = warp_max_u64(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long r = 0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) r = sh[w] > r ? sh[w] : r;
  return r;
}

template <typename TL, bool kScaled>
__global__ void narrow_kernel(const double* __restrict__ A, int64_t lda, int64_t n, TL* __restrict__ Nl,
                              int64_t ldn, const double* __restrict__ rinv, float* __restrict__ scale,
                              float* __restrict__ rowfac, int* __restrict__ rexp) {
  __shared__ float sh[32];
  __shared__ unsigned long long shb[32];
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double* row = A + i * lda;
    float s = 1.0f;
    if (kScaled) {
      float m = 0.0f;
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
        if (j != i) m = fmaxf(m, fabsf(__double2float_rn(row[j])));
      m = block_max_abs(m, sh);
      s = __fdiv_rn(m, 448.0f);
      if (s == 0.0f) s = 1.0f;
    }
    TL* out = Nl + i * ldn;
    unsigned long long mb = 0;  // max_j |a_ij| (all j, as IEEE bits)
    for (int64_t j = threadIdx.x; j < ldn; j += blockDim.x) {
      TL q;
      if (j < n) {
        const double a = row[j];
        const unsigned long long b = abs_bits(a);
        mb = b > mb ? b : mb;
        q = j != i ? narrow_encode<TL>(__double2float_rn(a), s) : narrow_encode<TL>(0.0f, 1.0f);
      } else {
        q = narrow_encode<TL>(0.0f, 1.0f);
      }
      out[j] = q;
    }
    if (rexp) {
      // exponent e with max_j |a_ij| < 2^e: the row scale of the split-float FP64 residual
      mb = block_max_bits(mb, shb);
      if (threadIdx.x == 0) {
        const double mx = __longlong_as_double(static_cast<long long>(mb));
        rexp[i] = (mx > 0.0 && isfinite(mx)) ? ilogb(mx) + 1 : 0;
      }
    }
    if (threadIdx.x == 0) {
      if (kScaled) scale[i] = s;
      rowfac[i] = __fmul_rn(__double2float_rn(rinv[i]), s);
    }
  }
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

cudaError_t launch_rhs(const double* B, int64_t n, double* b, unsigned long long* bnorm_bits, cudaStream_t s) {
  rhs_kernel<<<prep_blocks(n, kPrepThreads), kPrepThreads, 0, s>>>(B, n, b, bnorm_bits);
  return cudaGetLastError();
}

cudaError_t launch_pad_zero(double* M, int64_t n, int64_t ld, cudaStream_t s) {
  if (ld <= n) return cudaSuccess;
  pad_zero_kernel<<<prep_blocks(n, 1), 32, 0, s>>>(M, n, ld);
  return cudaGetLastError();
}

cudaError_t launch_narrow(Narrow kind, const double* A, int64_t lda, int64_t n, void* Nlow, int64_t ldn,
                          const double* rinv, float* scale, float* rowfac, int* rexp, cudaStream_t s) {
  const int blocks = prep_blocks(n, 1);
  switch (kind) {
    case Narrow::F32:
      narrow_kernel<float, false><<<blocks, kPrepThreads, 0, s>>>(A, lda, n, static_cast<float*>(Nlow), ldn, rinv,
                                                                  scale, rowfac, rexp);
      break;
    case Narrow::BF16:
      narrow_kernel<__nv_bfloat16, false><<<blocks, kPrepThreads, 0, s>>>(
          A, lda, n, static_cast<__nv_bfloat16*>(Nlow), ldn, rinv, scale, rowfac, rexp);
      break;
    case Narrow::E4M3:
      narrow_kernel<__nv_fp8_e4m3, true><<<blocks, kPrepThreads, 0, s>>>(
          A, lda, n, static_cast<__nv_fp8_e4m3*>(Nlow), ldn, rinv, scale, rowfac, rexp);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* A, int64_t lda, int64_t n, const double* b, const double* x,
                            unsigned long long* rmax_bits, cudaStream_t s) {
  residual_kernel<<<prep_blocks(n, 8), 256, 0, s>>>(A, lda, n, b, x, rmax_bits);
  return cudaGetLastError();
}

}  // namespace jac
