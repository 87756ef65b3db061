// Device-side building blocks of the persistent Jacobi kernels (sm_103a).
//
//  * mbarrier + cp.async.bulk (the TMA bulk-copy engine) for the shared-memory ring that streams
//    row blocks of the matrix, one elected producer warp per CTA;
//  * bounded waits (every spin reads %globaltimer and gives up with an error code, so a broken
//    invariant returns an error to the host instead of hanging the GPU);
//  * the grid-wide barrier of a cooperative launch (monotonic arrival counter, acquire/release).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace jac {

// Error codes a kernel writes to its control block (values of jacobi_status).
constexpr int kStatusOk = 0;
constexpr int kStatusNotConverged = 1;
constexpr int kStatusNonfinite = -3;
constexpr int kStatusTimeout = -6;

// Longest a device-side wait may spin before it reports kStatusTimeout (nanoseconds).  A healthy wait
// in these kernels lasts microseconds (one ring stage) to milliseconds (one phase of the largest
// system), so 4 s only ever fires on a broken invariant.
constexpr uint64_t kWaitLimitNs = 4000000000ull;

__device__ __forceinline__ int64_t i64min(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------------------- mbarrier

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the async proxy (the bulk-copy engine) and the CTA.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

// True once the phase with the given parity has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false if the limit expired.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// -------------------------------------------------------------------------- TMA bulk copy (1-D)

// Copy `bytes` (multiple of 16, both addresses 16-byte aligned) from global memory into this CTA's
// shared memory; completion is reported to `bar` as transaction bytes.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Orders this thread's earlier generic-proxy view of global memory before later async-proxy (bulk
// copy) accesses.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ------------------------------------------------------------------------------ global memory

__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned int* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// Order-free, NaN-propagating maximum of non-negative doubles: as unsigned 64-bit integers, the IEEE
// encodings of +0 .. +inf are increasing and every positive NaN is above +inf.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long abs_bits(float v) { return abs_bits(static_cast<double>(v)); }



__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid barrier of a cooperative launch, called by ONE thread per CTA after a CTA-wide barrier.
// `target` = (barrier index + 1) * gridDim.x.  Returns false if the wait timed out or another CTA
// reported an error through *status.
__device__ __forceinline__ bool grid_arrive_and_wait(unsigned int* counter, const int* status,
                                                     uint32_t target, uint64_t limit_ns = kWaitLimitNs) {
  __threadfence();
  atomicAdd(counter, 1u);
  if (ld_acquire_u32(counter) >= target) return true;
  const uint64_t t0 = global_timer_ns();
  while (ld_acquire_u32(counter) < target) {
    if (ld_volatile_i32(status) < 0) return false;
    if (global_timer_ns() - t0 > limit_ns) return false;
    __nanosleep(32);
  }
  __threadfence();
  return true;
}

// Named barrier among the first `threads` threads of the CTA.
__device__ __forceinline__ void named_barrier(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

}  // namespace jac
