// Batched solves of many independent dense systems of uneven size (the Jacobi iteration of Section 2,
// one system per CTA).
//
// Each system is small (n <= JACOBI_BATCH_MAX_N), so one CTA owns it for the whole solve: its iterates
// live in shared memory, its 8 warps stream the rows (RPW rows per warp at a time, 128-bit loads of the
// narrow copy, 128-bit loads of FP64 A where rows are 16-byte aligned, else 64-bit) and every sweep ends
// with one CTA barrier instead of a grid barrier.  The setup phase writes the narrow copy a row per warp
// with several loads per lane in flight, and computes the first inner sweep from the rounded values as it
// writes them, so that sweep does not read the copy back.  CTAs are persistent and take systems from a global atomic work queue, largest first, so
// systems of different sizes and sweep counts balance over the SMs.  This is the row-wise
// distribution of Section 3.1 applied at two levels: systems over SMs, rows over warps.
//
// Modes (per batch)
//   FP64      plain Jacobi in FP64, stopping when the relative residual of the previous iterate,
//             max_i |a_ii (x_i^(k) - x_i^(k-1))| / ||b||_inf, drops below tol (strict).
//   FP32/BF16 mixed precision: FP64 residual r = b - A x, inner Jacobi sweeps on the narrow copy of
//             the off-diagonal part of A written by the first phase, x += delta in FP64, until
//             ||b - A x||_inf / ||b||_inf <= tol.  For the zero start vector r = b: no matrix pass.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <new>
#include <vector>

#include "device_util.cuh"
#include "dot.cuh"
#include "solver.cuh"
#include "splitfloat.cuh"

namespace jac {
namespace {

constexpr int kBWarps = 8;
constexpr int kCopyLoads = 8;  // setup pass: FP64 loads per lane in flight (8-byte loads)
constexpr int kCopyPairs = 4;  // the same with 16-byte loads (rows 16-byte aligned)
constexpr int kBThreads = kBWarps * 32;
constexpr int kFL = 4;               // FP64 passes: lanes per row
constexpr int kFR = 32 / kFL;        // FP64 passes: rows per warp
constexpr int kFU = 4;               // FP64 passes: load steps per lane in flight

struct BatchSys {
  const double* A;  // row-major n x n, row stride n (read in place)
  const double* B;
  double* X;
  int64_t n;
  int64_t ldn;      // row stride of the narrow copy (multiple of 16)
  void* Nlow;       // narrow copy of the off-diagonal part (mixed modes)
  double* d;        // a_ii
  double* rinv;     // 1 / a_ii
  float* rowfac;    // (float) (1 / a_ii)
  float* c1;        // inner right-hand side
  int* rexp;        // split-float residual: per-row scale exponents (mixed modes)
  int64_t index;    // position in the caller's arrays
};

struct BatchParams {
  const BatchSys* sys;
  int64_t count;
  unsigned int* queue;
  jacobi_stats* stats;  // by caller index
  int64_t max_iter;
  double tol;
  int max_outer;
  int max_inner;
  float inner_rtol;
  int64_t smem_ld;      // length of each shared-memory vector
};

// Sum of RPW per-lane values over the warp, transposed: after the halving exchanges a lane holds one
// row's total (row = tr_row<RPW>(lane)); all lanes sharing the top log2(RPW) lane bits hold the same row.
template <int R, int OFF, typename Acc>
struct TR {
  static __device__ __forceinline__ Acc run(const Acc (&v)[R], int lane) {
    constexpr int H = R / 2;
    Acc w[H];
    const bool hi = lane & OFF;
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const Acc send = hi ? v[r] : v[r + H];
      const Acc keep = hi ? v[r + H] : v[r];
      w[r] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
    }
    return TR<H, OFF / 2, Acc>::run(w, lane);
  }
};
template <int OFF, typename Acc>
struct TR<1, OFF, Acc> {
  static __device__ __forceinline__ Acc run(const Acc (&v)[1], int lane) {
    Acc w = v[0];
#pragma unroll
    for (int o = OFF; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    return w;
  }
};
template <int R>
__device__ __forceinline__ int tr_row(int lane) {
  int row = 0;
  int bit = 4;
#pragma unroll
  for (int k = R; k > 1; k >>= 1, --bit) row = (row << 1) | ((lane >> bit) & 1);
  return row;
}
template <int R>
__device__ __forceinline__ bool tr_owner(int lane) {
  constexpr int low = 32 / R;  // lanes sharing one row's total
  return (lane & (low - 1)) == 0;
}

// Dot products of FP64 rows with the shared-memory FP64 vector x, L lanes per row: the warp takes rows
// [i0, i0 + 32 / L) and lane l works on row i0 + l / L.  The L lanes of a row split its columns (lane s
// takes the column pairs 2 s + 2 L t when rows are 16-byte aligned, else the columns s + L t), keep U
// steps of loads in flight and one FP64 accumulator each, and a log2(L)-level exchange sums them: fewer
// FP64 additions per row than the transposed reduction over 32 lanes below, which matters because the
// FP64 pipe is the residual's bound.  Every lane of the row returns the row's total.
template <int L, int U>
__device__ __forceinline__ double rows_fp64_lanes(const double* __restrict__ A, int64_t lda, int64_t n, int64_t i0,
                                                  const double* xs, int lane, bool al16) {
  const int s = lane & (L - 1);
  const int64_t i = i0 + lane / L;
  double acc = 0.0;
  if (i < n) {
    const double* a = A + i * lda;
    if (al16) {
      int64_t j = 2 * s;
      for (; j + 2 * L * (U - 1) + 1 < n; j += 2 * L * U) {
        double2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldg(reinterpret_cast<const double2*>(a + j + 2 * L * u));
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const double2 x = *reinterpret_cast<const double2*>(xs + j + 2 * L * u);
          acc = fma(v[u].x, x.x, acc);
          acc = fma(v[u].y, x.y, acc);
        }
      }
      for (; j < n; j += 2 * L) {
        if (j + 1 < n) {
          const double2 v = __ldg(reinterpret_cast<const double2*>(a + j));
          acc = fma(v.x, xs[j], acc);
          acc = fma(v.y, xs[j + 1], acc);
        } else {
          acc = fma(__ldg(a + j), xs[j], acc);
        }
      }
    } else {
      int64_t j = s;
      for (; j + L * (2 * U - 1) < n; j += 2 * L * U) {
        double v[2 * U];
#pragma unroll
        for (int u = 0; u < 2 * U; ++u) v[u] = __ldg(a + j + L * u);
#pragma unroll
        for (int u = 0; u < 2 * U; ++u) acc = fma(v[u], xs[j + L * u], acc);
      }
      for (; j < n; j += L) acc = fma(__ldg(a + j), xs[j], acc);
    }
  }
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// Dot products of FP64 rows [i0, i0 + RPW) (row stride lda) with x in the split-float arithmetic of
// splitfloat.cuh: lane l takes columns l + 32 t, each a_ij split (row scale 2^-e_i) as it is read, x as
// its two FP32 words in shared memory, float-float lane sums scaled back by 2^e_i before the FP64
// transposed reduction (the caller applies x's scale 2^g).
template <int RPW>
__device__ __forceinline__ double rows_split(const double* __restrict__ A, int64_t lda, int64_t n, int64_t i0,
                                             const float2* xs, const int* __restrict__ rexp, int lane) {
  FF acc[RPW];
  int sh[RPW];
  const int rows = static_cast<int>(i64min(RPW, n - i0));
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    acc[r] = FF{0.0f, 0.0f};
    sh[r] = r < rows ? rexp[i0 + r] : 0;
  }
  int64_t j = lane;
  for (; j + 96 < n; j += 128) {
    float2 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = xs[j + 32 * u];
#pragma unroll
    for (int r = 0; r < RPW; ++r)
      if (r < rows) {
        const double* a = A + (i0 + r) * lda + j;
        double av[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) av[u] = __ldg(a + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float h, l;
          split_scaled(av[u], sh[r], h, l);
          ff_fma(acc[r], h, l, x[u].x, x[u].y);
        }
        ff_renorm(acc[r]);
      }
  }
  for (; j < n; j += 32) {
    const float2 x = xs[j];
#pragma unroll
    for (int r = 0; r < RPW; ++r)
      if (r < rows) {
        float h, l;
        split_scaled(__ldg(A + (i0 + r) * lda + j), sh[r], h, l);
        ff_fma(acc[r], h, l, x.x, x.y);
      }
  }
  double dv[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) dv[r] = (static_cast<double>(acc[r].hi) + static_cast<double>(acc[r].lo)) * pow2(sh[r]);
  return TR<RPW, 16, double>::run(dv, lane);
}

// Narrow rows (16-byte segments, our own zero-padded copy, written earlier in this kernel: coherent
// loads) times the shared-memory FP32 vector x (zero beyond n).
template <typename TL, int RPW>
__device__ __forceinline__ float rows_narrow(const TL* __restrict__ N, int64_t ldn, int64_t n, int64_t i0,
                                             const float* xs, int lane) {
  constexpr int V = MatTraits<TL>::kVec;
  float acc[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) acc[r] = 0.0f;
  const int rows = static_cast<int>(i64min(RPW, n - i0));
  // two 16-byte segments of every row per lane and step (columns j and j + 32 V), loads before FMAs
  int64_t j = static_cast<int64_t>(lane) * V;
  for (; j + 32 * V < n; j += 64 * V) {
    float xv0[V], xv1[V];
#pragma unroll
    for (int q = 0; q < V / 4; ++q) {
      const float4 v0 = *reinterpret_cast<const float4*>(xs + j + 4 * q);
      const float4 v1 = *reinterpret_cast<const float4*>(xs + j + 32 * V + 4 * q);
      xv0[4 * q] = v0.x;
      xv0[4 * q + 1] = v0.y;
      xv0[4 * q + 2] = v0.z;
      xv0[4 * q + 3] = v0.w;
      xv1[4 * q] = v1.x;
      xv1[4 * q + 1] = v1.y;
      xv1[4 * q + 2] = v1.z;
      xv1[4 * q + 3] = v1.w;
    }
    uint4 m0[RPW], m1[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r)
      if (r < rows) {
        m0[r] = __ldcg(reinterpret_cast<const uint4*>(N + (i0 + r) * ldn + j));
        m1[r] = __ldcg(reinterpret_cast<const uint4*>(N + (i0 + r) * ldn + j + 32 * V));
      }
#pragma unroll
    for (int r = 0; r < RPW; ++r)
      if (r < rows) {
        seg_dot(acc[r], m0[r], xv0);
        seg_dot(acc[r], m1[r], xv1);
      }
  }
  for (; j < n; j += 32 * V) {
    float xv[V];
#pragma unroll
    for (int q = 0; q < V / 4; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(xs + j + 4 * q);
      xv[4 * q] = v.x;
      xv[4 * q + 1] = v.y;
      xv[4 * q + 2] = v.z;
      xv[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int r = 0; r < RPW; ++r)
      if (r < rows) {
        const uint4 m = __ldcg(reinterpret_cast<const uint4*>(N + (i0 + r) * ldn + j));
        seg_dot(acc[r], m, xv);
      }
  }
  return TR<RPW, 16, float>::run(acc, lane);
}

template <typename TL>
__device__ __forceinline__ TL encode_narrow(double a);
template <>
__device__ __forceinline__ float encode_narrow<float>(double a) {
  return __double2float_rn(a);
}
template <>
__device__ __forceinline__ __nv_bfloat16 encode_narrow<__nv_bfloat16>(double a) {
  return __float2bfloat16_rn(__double2float_rn(a));
}

// Two adjacent narrow values at p (p 2-element aligned: j even and ldn a multiple of 16).
__device__ __forceinline__ void store_pair(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ void store_pair(__nv_bfloat16* p, __nv_bfloat16 a, __nv_bfloat16 b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __halves2bfloat162(a, b);
}

// Maxima of two values over the CTA in one exchange (the barrier also publishes the shared-memory
// writes made before the call).
__device__ __forceinline__ void block_max2(unsigned long long& a, unsigned long long& b,
                                           unsigned long long (*sa)[kBWarps], unsigned long long (*sb)[kBWarps],
                                           int parity) {
  a = warp_max_u64(a);
  b = warp_max_u64(b);
  if ((threadIdx.x & 31) == 0) {
    sa[parity][threadIdx.x >> 5] = a;
    sb[parity][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  a = b = 0;
#pragma unroll
  for (int w = 0; w < kBWarps; ++w) {
    a = sa[parity][w] > a ? sa[parity][w] : a;
    b = sb[parity][w] > b ? sb[parity][w] : b;
  }
}

// Maximum over the CTA (the barrier also publishes the shared-memory writes made before the call).
__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long (*sred)[kBWarps],
                                                        int parity) {
  v = warp_max_u64(v);
  if ((threadIdx.x & 31) == 0) sred[parity][threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long m = 0;
#pragma unroll
  for (int w = 0; w < kBWarps; ++w) m = sred[parity][w] > m ? sred[parity][w] : m;
  return m;
}

// kMode: 0 = FP64 Jacobi, 1 = FP32 inner sweeps, 2 = BF16 inner sweeps.  kSplit (mixed modes): residuals
// with the split-float arithmetic instead of FP64 FMAs.
// MINB: CTAs per SM the register allocation must allow (1: as many registers as the compiler wants, about
// two CTAs per SM; 4: at most 64 registers, four CTAs and 32 warps per SM for more loads in flight).
template <int kMode, int RPW, bool kSplit, int MINB>
__global__ void __launch_bounds__(kBThreads, MINB) batch_kernel(BatchParams p) {
  using TL = typename std::conditional<kMode == 2, __nv_bfloat16, float>::type;
  extern __shared__ __align__(16) unsigned char bsmem[];
  __shared__ unsigned long long sred[2][kBWarps];   // phase-parity double buffer
  __shared__ unsigned long long sred2[2][kBWarps];
  __shared__ unsigned long long sph0[5][kBWarps];  // the setup phase's maxima
  __shared__ long long s_sys;
  double* xs0 = reinterpret_cast<double*>(bsmem);
  double* xs1 = xs0 + p.smem_ld;
  float* ds0 = reinterpret_cast<float*>(xs1 + p.smem_ld);
  float* ds1 = ds0 + p.smem_ld;
  float2* xss = reinterpret_cast<float2*>(ds1 + p.smem_ld);  // split words of x (split residual only)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (;;) {
    if (threadIdx.x == 0) s_sys = atomicAdd(p.queue, 1u);
    __syncthreads();
    const long long q = s_sys;
    __syncthreads();
    if (q >= p.count) break;
    const BatchSys S = p.sys[q];
    const int64_t n = S.n;
    const bool al16 = (n % 2 == 0) && (reinterpret_cast<uintptr_t>(S.A) % 16 == 0);

    // ---- phase 0: diagonal, ||b||, narrow copy (mixed modes); zero start vector
    unsigned long long bad = 0, bm = 0;
    for (int64_t i = threadIdx.x; i < n; i += kBThreads) {
      const double a = S.A[i * n + i];
      if (!isfinite(a))
        bad = bad ? bad : ((static_cast<unsigned long long>(i) << 8) | 3);
      else if (a == 0.0)
        bad = bad ? bad : ((static_cast<unsigned long long>(i) << 8) | 2);
      S.d[i] = a;
      const double ri = a != 0.0 ? __drcp_rn(a) : 0.0;
      S.rinv[i] = ri;
      S.rowfac[i] = __double2float_rn(ri);
      const unsigned long long bb = abs_bits(S.B[i]);
      bm = bb > bm ? bb : bm;
    }
    for (int64_t i = threadIdx.x; i < p.smem_ld; i += kBThreads) {
      xs0[i] = 0.0;
      xs1[i] = 0.0;
      ds0[i] = 0.0f;
      ds1[i] = 0.0f;
    }
    unsigned long long cm = 0;  // max_i |b_i / a_ii|: the iterate's scale for the split residual
    unsigned long long chg1 = 0, mag1 = 0;  // the first inner sweep's max |change| and max |delta|
    if (kMode != 0) {
      __syncthreads();  // reciprocals and zeroed vectors
      // the residual of the zero start vector (r = b) and c = r / a_ii, the inner iteration's start
      for (int64_t i = threadIdx.x; i < n; i += kBThreads) {
        const double r = S.B[i] - 0.0;
        const float c = static_cast<float>(r * S.rinv[i]);
        S.c1[i] = c;
        ds0[i] = c;
        if constexpr (kSplit) {
          const unsigned long long cb = abs_bits(S.B[i] * S.rinv[i]);
          cm = cb > cm ? cb : cm;
        }
      }
      __syncthreads();
      // the narrow copy, a row per warp, and with it the first inner sweep on the rounded values:
      // delta^(1)_i = c_i - (1/a_ii) sum_j fl(a_ij) c_j
      TL* Nl = static_cast<TL*>(S.Nlow);
      for (int64_t i = warp; i < n; i += kBWarps) {
        uint32_t mb = 0;
        float acc = 0.0f;
        // several loads per lane in flight before their conversions and stores; rows 16-byte aligned:
        // column pairs (16-byte loads, paired stores)
        if (al16) {
          for (int64_t j0 = 0; j0 < S.ldn; j0 += 64 * kCopyPairs) {
            double2 a[kCopyPairs];
#pragma unroll
            for (int u = 0; u < kCopyPairs; ++u) {
              const int64_t j = j0 + 2 * lane + 64 * u;
              a[u] = j < n ? __ldg(reinterpret_cast<const double2*>(S.A + i * n + j)) : double2{0.0, 0.0};
            }
#pragma unroll
            for (int u = 0; u < kCopyPairs; ++u) {
              const int64_t j = j0 + 2 * lane + 64 * u;
              if (j < S.ldn) {
                if constexpr (kSplit) mb = max(mb, max(abs_hi(a[u].x), abs_hi(a[u].y)));
                const TL e0 = (j < n && j != i) ? encode_narrow<TL>(a[u].x) : TL(0.0f);
                const TL e1 = (j + 1 < n && j + 1 != i) ? encode_narrow<TL>(a[u].y) : TL(0.0f);
                store_pair(Nl + i * S.ldn + j, e0, e1);
                const float2 c = *reinterpret_cast<const float2*>(ds0 + j);
                acc = fmaf(static_cast<float>(e0), c.x, acc);
                acc = fmaf(static_cast<float>(e1), c.y, acc);
              }
            }
          }
        } else {
          for (int64_t j0 = 0; j0 < S.ldn; j0 += 32 * kCopyLoads) {
            double a[kCopyLoads];
#pragma unroll
            for (int u = 0; u < kCopyLoads; ++u) {
              const int64_t j = j0 + lane + 32 * u;
              a[u] = j < n ? __ldg(S.A + i * n + j) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kCopyLoads; ++u) {
              const int64_t j = j0 + lane + 32 * u;
              if (j < S.ldn) {
                if constexpr (kSplit) mb = max(mb, abs_hi(a[u]));
                const TL e = (j < n && j != i) ? encode_narrow<TL>(a[u]) : TL(0.0f);
                Nl[i * S.ldn + j] = e;
                acc = fmaf(static_cast<float>(e), ds0[j], acc);
              }
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if constexpr (kSplit) {
          mb = __reduce_max_sync(0xffffffffu, mb);
          if (lane == 0) S.rexp[i] = split_exponent_hi(mb);
        }
        if (lane == 0) {
          const float v = fmaf(-S.rowfac[i], acc, S.c1[i]);
          ds1[i] = v;
          const unsigned long long a1 = abs_bits(v - ds0[i]), a2 = abs_bits(v);
          chg1 = a1 > chg1 ? a1 : chg1;
          mag1 = a2 > mag1 ? a2 : mag1;
        }
      }
    }
    // the setup's maxima in one exchange; the first failing row decides (smallest index)
    if (bad) bad = ~bad;  // so that the max picks the smallest key
    {
      unsigned long long v[5] = {bad, bm, cm, chg1, mag1};
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] = warp_max_u64(v[k]);
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) sph0[k][warp] = v[k];
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        v[k] = 0;
#pragma unroll
        for (int w = 0; w < kBWarps; ++w) v[k] = sph0[k][w] > v[k] ? sph0[k][w] : v[k];
      }
      bad = v[0];
      bm = v[1];
      cm = v[2];
      chg1 = v[3];
      mag1 = v[4];
    }
    const unsigned long long badmax = bad;
    const unsigned long long bmax_bits = bm;
    const double bnorm = __longlong_as_double(static_cast<long long>(bmax_bits));
    int xg = 0;
    if constexpr (kSplit) xg = split_exponent(cm);
    jacobi_stats st{};
    st.rel_residual = __longlong_as_double(0x7FF8000000000000ll);
    int status = kStatusNotConverged;
    int parity = 1;
    int cur = 0;  // FP64 iterate buffer (0: xs0)
    if (badmax) {
      const unsigned long long key = ~badmax;
      status = (key & 0xFF) == 2 ? JACOBI_ERR_ZERO_DIAGONAL : JACOBI_ERR_NONFINITE;
    } else if (kMode == 0) {
      // ---- plain FP64 Jacobi, residual-of-previous-iterate stop
      int64_t k = 1;
      for (;; ++k, parity ^= 1) {
        const double* xc = cur ? xs1 : xs0;
        double* xn = cur ? xs0 : xs1;
        unsigned long long mx = 0;
        for (int64_t i0 = static_cast<int64_t>(warp) * kFR; i0 < n; i0 += static_cast<int64_t>(kBWarps) * kFR) {
          const double dot = rows_fp64_lanes<kFL, kFU>(S.A, n, n, i0, xc, lane, al16);
          const int64_t i = i0 + lane / kFL;
          if ((lane & (kFL - 1)) == 0 && i < n) {
            const double xo = xc[i];
            const double sdot = fma(-S.d[i], xo, dot);
            const double xi = (S.B[i] - sdot) * S.rinv[i];
            xn[i] = xi;
            const unsigned long long v = abs_bits(S.d[i] * (xi - xo));
            mx = v > mx ? v : mx;
          }
        }
        const double delta = __longlong_as_double(static_cast<long long>(block_max(mx, sred, parity))) / bnorm;
        st.final_delta = delta;
        st.sweeps = k;
        cur ^= 1;
        if (!isfinite(delta)) {
          status = kStatusNonfinite;
          break;
        }
        if (delta < p.tol) {
          status = kStatusOk;
          break;
        }
        if (k >= p.max_iter) break;
      }
    } else {
      // ---- mixed precision: FP64 residual, narrow inner sweeps, FP64 update
      const TL* Nl = static_cast<const TL*>(S.Nlow);
      int64_t outer = 0, inner_total = 0;
      bool first = true;
      for (;;) {
        // residual of the current iterate; for the zero start vector r = b (c and the first inner sweep
        // were computed by the setup phase) and max |r_i| = ||b||
        const double* xc = cur ? xs1 : xs0;
        unsigned long long mr = bmax_bits;
        if (!first) {
          if constexpr (kSplit) {
            for (int64_t i = threadIdx.x; i < p.smem_ld; i += kBThreads) xss[i] = i < n ? split_x(xc[i], xg) : float2{};
            __syncthreads();
          }
          mr = 0;
          // rows of the residual: RPW rows per warp (split-float), or kFR (FP64 FMAs, kFL lanes per row)
          constexpr int64_t kRows = kSplit ? RPW : kFR;
          for (int64_t i0 = static_cast<int64_t>(warp) * kRows; i0 < n; i0 += static_cast<int64_t>(kBWarps) * kRows) {
            double dot;
            int64_t i;
            bool owner;
            if constexpr (kSplit) {
              dot = rows_split<RPW>(S.A, n, n, i0, xss, S.rexp, lane) * pow2(xg);
              i = i0 + tr_row<RPW>(lane);
              owner = tr_owner<RPW>(lane);
            } else {
              dot = rows_fp64_lanes<kFL, kFU>(S.A, n, n, i0, xc, lane, al16);
              i = i0 + lane / kFL;
              owner = (lane & (kFL - 1)) == 0;
            }
            if (owner && i < n) {
              const double r = S.B[i] - dot;
              const float c = static_cast<float>(r * S.rinv[i]);
              S.c1[i] = c;
              ds0[i] = c;
              const unsigned long long vr = abs_bits(r);
              mr = vr > mr ? vr : mr;
            }
          }
          mr = block_max(mr, sred, parity);
          parity ^= 1;
        }
        const bool pre = first;  // the first inner sweep of this outer step is done (setup phase)
        first = false;
        ++outer;
        const double rho = __longlong_as_double(static_cast<long long>(mr)) / bnorm;
        st.rel_residual = rho;
        if (!isfinite(rho)) {
          status = kStatusNonfinite;
          break;
        }
        if (rho <= p.tol) {
          status = kStatusOk;
          break;
        }
        if (outer >= p.max_outer || inner_total >= p.max_iter) break;
        // inner sweeps: delta^(m) = c1 - (1/a_ii) * (N delta^(m-1)), candidate x + delta in FP64
        int dcur = 0;
        const double* xcc = cur ? xs1 : xs0;
        double* xalt = cur ? xs0 : xs1;
        int64_t m0 = 1;
        bool more = true;
        if (pre) {
          // delta^(1) is in ds1 (cur is 0 here)
          const double chg = __longlong_as_double(static_cast<long long>(chg1));
          const double mag = __longlong_as_double(static_cast<long long>(mag1));
          ++inner_total;
          st.final_delta = chg;
          dcur = 1;
          if (!isfinite(chg) || !isfinite(mag)) {
            status = kStatusNonfinite;
            break;
          }
          more = !(chg <= static_cast<double>(p.inner_rtol) * mag || 1 >= p.max_inner || inner_total >= p.max_iter);
          m0 = 2;
        }
        for (int64_t m = m0; more; ++m) {
          const float* dc = dcur ? ds1 : ds0;
          float* dn = dcur ? ds0 : ds1;
          // maxima as FP32 bits (non-negative floats order like their bits; NaN above infinity), widened
          // once for the exchange
          unsigned int fchg = 0, fmag = 0;
          for (int64_t i0 = static_cast<int64_t>(warp) * RPW; i0 < n; i0 += static_cast<int64_t>(kBWarps) * RPW) {
            const float dot = rows_narrow<TL, RPW>(Nl, S.ldn, n, i0, dc, lane);
            const int64_t i = i0 + tr_row<RPW>(lane);
            if (tr_owner<RPW>(lane) && i < n) {
              const float v = fmaf(-S.rowfac[i], dot, S.c1[i]);
              const float old = dc[i];
              dn[i] = v;
              const unsigned int a1 = __float_as_uint(fabsf(v - old)), a2 = __float_as_uint(fabsf(v));
              fchg = a1 > fchg ? a1 : fchg;
              fmag = a2 > fmag ? a2 : fmag;
            }
          }
          unsigned long long mchg = abs_bits(__uint_as_float(fchg)), mmag = abs_bits(__uint_as_float(fmag));
          block_max2(mchg, mmag, sred, sred2, parity);
          const double chg = __longlong_as_double(static_cast<long long>(mchg));
          const double mag = __longlong_as_double(static_cast<long long>(mmag));
          parity ^= 1;
          ++inner_total;
          st.final_delta = chg;
          dcur ^= 1;
          if (!isfinite(chg) || !isfinite(mag)) {
            status = kStatusNonfinite;
            break;
          }
          if (chg <= static_cast<double>(p.inner_rtol) * mag || m >= p.max_inner || inner_total >= p.max_iter)
            break;
        }
        if (status == kStatusNonfinite) break;
        // x + delta becomes the current iterate (delta: the last sweep's, in ds[dcur])
        {
          const float* df = dcur ? ds1 : ds0;
          for (int64_t i = threadIdx.x; i < n; i += kBThreads) xalt[i] = xcc[i] + static_cast<double>(df[i]);
          __syncthreads();
        }
        cur ^= 1;
      }
      st.sweeps = inner_total;
      st.outer_steps = outer;
    }
    // ---- output (the current iterate) and the record
    const double* xr = cur ? xs1 : xs0;
    for (int64_t i = threadIdx.x; i < n; i += kBThreads) S.X[i] = xr[i];
    if (threadIdx.x == 0) {
      st.status = status;
      st.converged = status == kStatusOk;
      p.stats[S.index] = st;
    }
    __syncthreads();
  }
}

using BatchKernel = void (*)(BatchParams);

template <int M, bool kSplit, int MINB>
BatchKernel pick_rpw(int rpw) {
  switch (rpw) {
    case 1: return batch_kernel<M, 1, kSplit, MINB>;
    case 2: return batch_kernel<M, 2, kSplit, MINB>;
    case 8: return batch_kernel<M, 8, kSplit, MINB>;
    default: return batch_kernel<M, 4, kSplit, MINB>;
  }
}

template <int MINB>
BatchKernel pick_occ(int precision, int rpw, bool split) {
  if (precision == JACOBI_FP64) return pick_rpw<0, false, MINB>(rpw);
  if (precision == JACOBI_FP32_IR) return split ? pick_rpw<1, true, MINB>(rpw) : pick_rpw<1, false, MINB>(rpw);
  return split ? pick_rpw<2, true, MINB>(rpw) : pick_rpw<2, false, MINB>(rpw);
}

// ctas_per_sm >= 3 asks for the register-limited build (four CTAs per SM can be resident).
BatchKernel pick_kernel(int precision, int rpw, bool split, int ctas_per_sm) {
  return ctas_per_sm >= 3 ? pick_occ<4>(precision, rpw, split) : pick_occ<1>(precision, rpw, split);
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace jac

using namespace jac;

struct jacobi_batch {
  int64_t count = 0;
  int precision = JACOBI_FP32_IR;
  int rpw = 4;
  int cps = 0;  // requested CTAs per SM (0: all that fit)
  bool split = false;
  int grid = 0;
  size_t smem = 0;
  int64_t smem_ld = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  bool own_ws = false;
  char* ws = nullptr;
  BatchSys* dsys = nullptr;
  unsigned int* queue = nullptr;
  jacobi_stats* stats = nullptr;
  int max_outer = 30, max_inner = 1000;
  float inner_rtol = 1.0f / 16384;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t g_max_iter = -1;
  double g_tol = -1.0;
};

namespace {

struct BatchLayout {
  size_t sys, queue, stats, total;
  std::vector<size_t> per;  // start of each system's region
};

size_t narrow_bytes(int precision) { return precision == JACOBI_FP32_IR ? 4 : precision == JACOBI_BF16_IR ? 2 : 0; }

BatchLayout batch_layout(const jacobi_batch_desc* d) {
  BatchLayout L;
  size_t o = 0;
  L.sys = o;
  o = align256(o + static_cast<size_t>(d->count) * sizeof(BatchSys));
  L.queue = o;
  o = align256(o + sizeof(unsigned int));
  L.stats = o;
  o = align256(o + static_cast<size_t>(d->count) * sizeof(jacobi_stats));
  const size_t es = narrow_bytes(d->precision);
  L.per.resize(static_cast<size_t>(d->count));
  for (int64_t k = 0; k < d->count; ++k) {
    const int64_t n = d->n[k];
    const int64_t ld = round_up(n, kLdAlign);
    L.per[static_cast<size_t>(k)] = o;
    o = align256(o + static_cast<size_t>(n) * ld * es);  // narrow copy
    o = align256(o + static_cast<size_t>(ld) * (8 + 8 + 4 + 4 + 4));  // d, rinv, rowfac, c1, rexp
  }
  L.total = o;
  return L;
}

int batch_validate(const jacobi_batch_desc* d) {
  if (!d || d->count < 1 || !d->n || !d->A || !d->B || !d->X) return JACOBI_ERR_INVALID_ARG;
  if (d->precision != JACOBI_FP64 && d->precision != JACOBI_FP32_IR && d->precision != JACOBI_BF16_IR)
    return JACOBI_ERR_INVALID_ARG;
  if (d->rows_per_warp != 0 && d->rows_per_warp != 1 && d->rows_per_warp != 2 && d->rows_per_warp != 4 &&
      d->rows_per_warp != 8)
    return JACOBI_ERR_INVALID_ARG;
  for (int64_t k = 0; k < d->count; ++k) {
    if (d->n[k] < 1 || d->n[k] > JACOBI_BATCH_MAX_N) return JACOBI_ERR_INVALID_ARG;
    if (!d->A[k] || !d->B[k] || !d->X[k]) return JACOBI_ERR_INVALID_ARG;
  }
  return JACOBI_OK;
}

}  // namespace

extern "C" {

int jacobi_batch_workspace_size(const jacobi_batch_desc* d, size_t* bytes) {
  if (!bytes) return JACOBI_ERR_INVALID_ARG;
  const int v = batch_validate(d);
  if (v != JACOBI_OK) return v;
  *bytes = batch_layout(d).total;
  return JACOBI_OK;
}

int jacobi_batch_create(const jacobi_batch_desc* d, jacobi_batch** out) {
  if (!out) return JACOBI_ERR_INVALID_ARG;
  *out = nullptr;
  const int v = batch_validate(d);
  if (v != JACOBI_OK) return v;
  jacobi_batch* b = new (std::nothrow) jacobi_batch();
  if (!b) return JACOBI_ERR_OUT_OF_MEMORY;
  b->count = d->count;
  b->precision = d->precision;
  b->rpw = d->rows_per_warp ? d->rows_per_warp : 4;
  b->split = (d->flags & JACOBI_FLAG_SPLIT_RESIDUAL) && d->precision != JACOBI_FP64;
  b->stream = static_cast<cudaStream_t>(d->stream);
  if (d->max_outer > 0) b->max_outer = d->max_outer;
  if (d->max_inner > 0) b->max_inner = d->max_inner;
  if (d->inner_rtol > 0) b->inner_rtol = static_cast<float>(d->inner_rtol);
  const BatchLayout L = batch_layout(d);
  auto fail = [&](int st) {
    jacobi_batch_destroy(b);
    return st;
  };
  if (d->workspace) {
    if (d->workspace_bytes < L.total || reinterpret_cast<uintptr_t>(d->workspace) % 256) return fail(JACOBI_ERR_INVALID_ARG);
    b->ws = static_cast<char*>(d->workspace);
  } else {
    if (cudaMalloc(&b->ws, L.total) != cudaSuccess) return fail(JACOBI_ERR_OUT_OF_MEMORY);
    b->own_ws = true;
  }
  // systems largest first: the queue hands out the long solves early and the short ones fill the tail
  std::vector<int64_t> order(static_cast<size_t>(d->count));
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t c) { return d->n[a] > d->n[c]; });
  std::vector<BatchSys> host(static_cast<size_t>(d->count));
  const size_t es = narrow_bytes(d->precision);
  int64_t nmax = 0;
  for (size_t q = 0; q < order.size(); ++q) {
    const int64_t k = order[q];
    const int64_t n = d->n[k];
    const int64_t ld = round_up(n, kLdAlign);
    nmax = std::max(nmax, n);
    char* base = b->ws + L.per[static_cast<size_t>(k)];
    BatchSys s{};
    s.A = d->A[k];
    s.B = d->B[k];
    s.X = d->X[k];
    s.n = n;
    s.ldn = ld;
    s.Nlow = es ? base : nullptr;
    char* v = base + align256(static_cast<size_t>(n) * ld * es);
    s.d = reinterpret_cast<double*>(v);
    s.rinv = s.d + ld;
    s.rowfac = reinterpret_cast<float*>(s.rinv + ld);
    s.c1 = s.rowfac + ld;
    s.rexp = reinterpret_cast<int*>(s.c1 + ld);
    s.index = k;
    host[q] = s;
  }
  b->dsys = reinterpret_cast<BatchSys*>(b->ws + L.sys);
  b->queue = reinterpret_cast<unsigned int*>(b->ws + L.queue);
  b->stats = reinterpret_cast<jacobi_stats*>(b->ws + L.stats);
  if (cudaMemcpyAsync(b->dsys, host.data(), host.size() * sizeof(BatchSys), cudaMemcpyHostToDevice, b->stream) !=
      cudaSuccess)
    return fail(JACOBI_ERR_CUDA);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(JACOBI_ERR_CUDA);
  b->smem_ld = round_up(nmax, kLdAlign);
  b->smem = static_cast<size_t>(b->smem_ld) * (2 * sizeof(double) + 2 * sizeof(float) + (b->split ? sizeof(float2) : 0));
  b->cps = d->ctas_per_sm;
  BatchKernel kern = pick_kernel(b->precision, b->rpw, b->split, b->cps);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(b->smem)) != cudaSuccess)
    return fail(JACOBI_ERR_CUDA);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBThreads, b->smem) != cudaSuccess || per_sm < 1)
    return fail(JACOBI_ERR_CUDA);
  if (d->ctas_per_sm > 0 && d->ctas_per_sm < per_sm) per_sm = d->ctas_per_sm;
  b->grid = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(per_sm) * sms, d->count));
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) return fail(JACOBI_ERR_CUDA);
  *out = b;
  return JACOBI_OK;
}

int jacobi_batch_solve_async(jacobi_batch* b, int64_t max_iter, double tol) {
  if (!b || max_iter < 1 || !(tol > 0.0) || !std::isfinite(tol)) return JACOBI_ERR_INVALID_ARG;
  if (!b->exec || b->g_max_iter != max_iter || b->g_tol != tol) {
    // capture the solve (queue reset + the persistent kernel) once per (max_iter, tol); later calls
    // replay the instantiated graph
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (b->graph) {
      cudaGraphDestroy(b->graph);
      b->graph = nullptr;
    }
    BatchParams p{};
    p.sys = b->dsys;
    p.count = b->count;
    p.queue = b->queue;
    p.stats = b->stats;
    p.max_iter = max_iter;
    p.tol = tol;
    p.max_outer = b->max_outer;
    p.max_inner = b->max_inner;
    p.inner_rtol = b->inner_rtol;
    p.smem_ld = b->smem_ld;
    BatchKernel kern = pick_kernel(b->precision, b->rpw, b->split, b->cps);
    if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return JACOBI_ERR_CUDA;
    cudaMemsetAsync(b->queue, 0, sizeof(unsigned int), b->capture);
    void* args[] = {&p};
    const cudaError_t le = cudaLaunchKernel(reinterpret_cast<const void*>(kern), dim3(b->grid), dim3(kBThreads), args,
                                            b->smem, b->capture);
    const cudaError_t ce = cudaStreamEndCapture(b->capture, &b->graph);
    if (le != cudaSuccess || ce != cudaSuccess) return JACOBI_ERR_CUDA;
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return JACOBI_ERR_CUDA;
    b->g_max_iter = max_iter;
    b->g_tol = tol;
  }
  if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return JACOBI_ERR_CUDA;
  return JACOBI_OK;
}

int jacobi_batch_stats(jacobi_batch* b, jacobi_stats* stats) {
  if (!b || !stats) return JACOBI_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(stats, b->stats, static_cast<size_t>(b->count) * sizeof(jacobi_stats), cudaMemcpyDeviceToHost,
                      b->stream) != cudaSuccess)
    return JACOBI_ERR_CUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return JACOBI_ERR_CUDA;
  return JACOBI_OK;
}

int jacobi_batch_grid(jacobi_batch* b) { return b ? b->grid : 0; }

void jacobi_batch_destroy(jacobi_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->own_ws && b->ws) cudaFree(b->ws);
  delete b;
}

int jacobi_batch_solve(int64_t count, const int64_t* n, const double* const* A, const double* const* B,
                       double* const* X_out, double tol, int64_t max_iter, int32_t precision, jacobi_stats* stats) {
  if (count < 1 || !n || !A || !B || !X_out) return JACOBI_ERR_INVALID_ARG;
  jacobi_batch_desc d{};
  d.count = count;
  d.n = n;
  d.A = A;
  d.B = B;
  d.X = X_out;
  d.precision = precision;
  // the autotuner's shape for thousands of systems of a few hundred unknowns
  d.rows_per_warp = 4;
  d.ctas_per_sm = 4;
  d.inner_rtol = 1.0 / 1024;
  jacobi_batch* b = nullptr;
  int st = jacobi_batch_create(&d, &b);
  if (st != JACOBI_OK) return st;
  std::vector<jacobi_stats> local;
  jacobi_stats* out = stats;
  if (!out) {
    local.resize(static_cast<size_t>(count));
    out = local.data();
  }
  st = jacobi_batch_solve_async(b, max_iter, tol);
  if (st == JACOBI_OK) st = jacobi_batch_stats(b, out);
  jacobi_batch_destroy(b);
  if (st != JACOBI_OK) return st;
  // the worst outcome over the systems: an error, else a system that hit its cap, else converged
  int worst = JACOBI_OK;
  for (int64_t k = 0; k < count; ++k) {
    const int sk = out[k].status;
    if (sk < 0) {
      if (worst >= 0 || sk < worst) worst = sk;  // an error outranks any warning
    } else if (sk > 0 && worst == JACOBI_OK) {
      worst = sk;
    }
  }
  return worst;
}

}  // extern "C"
