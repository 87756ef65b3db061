// Measured arithmetic rates of this GPU's CUDA cores, the denominators of the FP64-FMA and FP32 bounds
// that the FP64 sweeps, the FP64 residual passes and the split-float residual are held to.
//
// Each thread runs CH independent FMA chains, so that the issue of the FMA pipe, not its latency, limits
// the rate; the grid holds every SM with BPS blocks of kPeakThreads threads.  Two operand forms are timed:
// the recurrence x <- x * m + c (|m| < 1, values stay finite) and the dot-product form acc <- a * b + acc
// with per-chain a and b, the form of the solver's row dot products.  On GB300 the FP64 pipe reaches its
// 2 FMAs per clock per SM only in the second form with 4 chains (the recurrence stops near 0.84 of it).
// Several (form, CH, BPS) shapes are timed, each launch after an untimed one on the same stream (CUDA
// events), and the best rate is reported.
#include <cuda_runtime.h>

#include "solver.cuh"

namespace jac {
namespace {

constexpr int kPeakThreads = 256;

template <typename T, int CH>
__global__ void __launch_bounds__(kPeakThreads) fma_rate_kernel(int64_t iters, T m, T c, T* sink) {
  T x[CH];
#pragma unroll
  for (int u = 0; u < CH; ++u) x[u] = static_cast<T>(threadIdx.x + u) * static_cast<T>(1e-3);
  for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < CH; ++u) x[u] = fma(x[u], m, c);
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < CH; ++u) s += x[u];
  if (s == static_cast<T>(-1.5)) sink[0] = s;  // never true; keeps the chains live
}

template <typename T, int CH>
__global__ void __launch_bounds__(kPeakThreads) fma_dot_kernel(int64_t iters, T m, T c, T* sink) {
  T acc[CH], a[CH], b[CH];
#pragma unroll
  for (int u = 0; u < CH; ++u) {
    acc[u] = static_cast<T>(0);
    a[u] = static_cast<T>(threadIdx.x + u) * c;
    b[u] = m + static_cast<T>(u) * static_cast<T>(1e-3);
  }
  for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
    for (int u = 0; u < CH; ++u) acc[u] = fma(a[u], b[u], acc[u]);
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < CH; ++u) s += acc[u];
  if (s == static_cast<T>(-1.5)) sink[0] = s;  // never true (every term is non-negative); keeps the chains live
}

template <typename T, int CH, bool kDot>
cudaError_t time_rate_shape(int64_t iters, int bps, cudaStream_t s, double* per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = sms * bps;
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  const T m = static_cast<T>(0.999999), c = static_cast<T>(1e-7);
  auto kern = kDot ? fma_dot_kernel<T, CH> : fma_rate_kernel<T, CH>;
  kern<<<grid, kPeakThreads, 0, s>>>(iters / 4 + 1, m, c, nullptr);
  cudaEventRecord(a, s);
  kern<<<grid, kPeakThreads, 0, s>>>(iters, m, c, nullptr);
  cudaEventRecord(b, s);
  e = cudaEventSynchronize(b);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  const double fmas = static_cast<double>(grid) * kPeakThreads * CH * static_cast<double>(iters);
  *per_s = ms > 0.0f ? fmas / (static_cast<double>(ms) * 1e-3) : 0.0;
  return cudaSuccess;
}

// Best over both forms, 4 or 16 chains per thread and 4 or 8 blocks per SM (the same FMA count per
// thread each time).
template <typename T>
cudaError_t time_rate(int64_t iters, cudaStream_t s, double* per_s) {
  double best = 0.0, r = 0.0;
  for (int bps : {4, 8}) {
    cudaError_t e = time_rate_shape<T, 4, false>(iters * 4, bps, s, &r);
    if (e != cudaSuccess) return e;
    best = r > best ? r : best;
    e = time_rate_shape<T, 16, false>(iters, bps, s, &r);
    if (e != cudaSuccess) return e;
    best = r > best ? r : best;
    e = time_rate_shape<T, 4, true>(iters * 4, bps, s, &r);
    if (e != cudaSuccess) return e;
    best = r > best ? r : best;
    e = time_rate_shape<T, 16, true>(iters, bps, s, &r);
    if (e != cudaSuccess) return e;
    best = r > best ? r : best;
  }
  *per_s = best;
  return cudaSuccess;
}

}  // namespace
}  // namespace jac

extern "C" int jacobi_measure_fma_rates(int64_t iters, double* fp64_fma_per_s, double* fp32_fma_per_s,
                                        void* stream) {
  if (iters < 1 || !fp64_fma_per_s || !fp32_fma_per_s) return JACOBI_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (jac::time_rate<double>(iters, s, fp64_fma_per_s) != cudaSuccess) return JACOBI_ERR_CUDA;
  // the FP32 pipe is about 64 times faster: run 64 times the iterations for a comparable duration
  if (jac::time_rate<float>(iters * 64, s, fp32_fma_per_s) != cudaSuccess) return JACOBI_ERR_CUDA;
  return JACOBI_OK;
}
