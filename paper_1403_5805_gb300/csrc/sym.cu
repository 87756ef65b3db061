// Symmetric A stored once for the narrow inner sweeps of the mixed-precision refinement.
//
// The inner sweep delta_i <- c1_i - f_i sum_{j != i} a_ij delta_j (f_i = 1/a_ii, Section 2's update of
// A delta = r) reads the off-diagonal part of A in a narrow format.  When A is symmetric only the tiles on
// and above the diagonal are stored (128 x 128 each, packed in row-of-tiles order), and every off-diagonal
// tile (I, J), I < J, serves two row blocks in one read: its row dots sum_{j in J} a_ij delta_j go to the
// rows of block I and its column dots sum_{i in I} a_ij delta_i to the rows of block J (a_ji = a_ij).
// Diagonal tiles hold the full symmetric block (zero diagonal) and give row dots only.  The partial sums
// land in fixed slots, P[I][K] for the contribution of tile (I, K) or (K, I) to block I, and a second
// kernel adds each row's nt slots in slot order, so the result does not depend on scheduling.
//
// The FP64 residual r = b - A x reads the full FP64 A (the refinement's accuracy comes from it).
#include <cuda_bf16.h>

#include <cstdint>

#include "device_util.cuh"
#include "f64tof32.cuh"
#include "solver.cuh"
#include "sym.cuh"

namespace jac {
namespace {

constexpr int kSymThreads = 256;  // 8 warps x 16 rows of a tile; lane l holds columns 4 l .. 4 l + 3

template <typename TL>
__device__ __forceinline__ TL sym_encode(double a);
template <>
__device__ __forceinline__ float sym_encode<float>(double a) {
  return f64_to_f32_rn(a);
}
template <>
__device__ __forceinline__ __nv_bfloat16 sym_encode<__nv_bfloat16>(double a) {
  return __float2bfloat16_rn(f64_to_f32_rn(a));  // FP64 -> FP32 -> BF16, each to nearest even
}

// Four consecutive narrow entries of a tile row as FP32.
__device__ __forceinline__ void sym_load4(const float* p, float (&v)[4]) {
  const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
  v[3] = q.w;
}
__device__ __forceinline__ void sym_load4(const __nv_bfloat16* p, float (&v)[4]) {
  const uint2 q = __ldcs(reinterpret_cast<const uint2*>(p));
  v[0] = __uint_as_float(q.x << 16);
  v[1] = __uint_as_float(q.x & 0xFFFF0000u);
  v[2] = __uint_as_float(q.y << 16);
  v[3] = __uint_as_float(q.y & 0xFFFF0000u);
}

// Packed index t of tile (I, J), I <= J, and its inverse.
__device__ __forceinline__ int64_t tile_start(int64_t I, int64_t nt) { return I * nt - I * (I - 1) / 2; }
__device__ __forceinline__ void tile_coords(int64_t t, int64_t nt, int64_t& I, int64_t& J) {
  int64_t lo = 0, hi = nt - 1;  // last I with tile_start(I) <= t
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (tile_start(mid, nt) <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  I = lo;
  J = I + (t - tile_start(I, nt));
}

// One CTA per packed tile: the off-diagonal entries of A's rows of block I and columns of block J
// (zero on the diagonal and outside n), rounded to the narrow type; diagonal tiles also write the FP32
// row factor f_i = fl32(1 / a_ii) of their rows.
template <typename TL>
__global__ void sym_pack_kernel(const double* __restrict__ A, int64_t lda, int64_t n, int64_t nt,
                                const double* __restrict__ rinv, TL* __restrict__ tiles, float* __restrict__ rowfac) {
  int64_t I, J;
  tile_coords(blockIdx.x, nt, I, J);
  TL* T = tiles + static_cast<int64_t>(blockIdx.x) * kSymTile * kSymTile;
  for (int e = threadIdx.x; e < kSymTile * kSymTile; e += blockDim.x) {
    const int64_t i = I * kSymTile + e / kSymTile, j = J * kSymTile + e % kSymTile;
    const double a = (i < n && j < n && i != j) ? A[i * lda + j] : 0.0;
    T[e] = sym_encode<TL>(a);
  }
  if (I == J && threadIdx.x < kSymTile) {
    const int64_t i = I * kSymTile + threadIdx.x;
    if (i < n) rowfac[i] = __double2float_rn(rinv[i]);
  }
}

// Transposed sum over the 32 lanes of 16 per-lane values (one per row): afterwards the two lanes 2 r and
// 2 r + 1 ... hold row r's total, r = bits 4..1 of the lane (fixed order of additions).
template <int R, int OFF>
struct SymTR {
  static __device__ __forceinline__ float run(const float (&v)[R], int lane) {
    constexpr int H = R / 2;
    float w[H];
    const bool hi = lane & OFF;
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const float send = hi ? v[q] : v[q + H];
      const float keep = hi ? v[q + H] : v[q];
      w[q] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
    }
    return SymTR<H, OFF / 2>::run(w, lane);
  }
};
template <int OFF>
struct SymTR<1, OFF> {
  static __device__ __forceinline__ float run(const float (&v)[1], int lane) {
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], OFF);
  }
};
__device__ __forceinline__ int symtr_row(int lane) {  // row index held by this lane after SymTR<16, 16>
  return ((lane >> 4) & 1) << 3 | ((lane >> 3) & 1) << 2 | ((lane >> 2) & 1) << 1 | ((lane >> 1) & 1);
}

// One CTA per packed tile (I, J): row dots of its 128 rows against delta of block J into P[I][J], and (I < J)
// column dots against delta of block I into P[J][I].
template <typename TL>
__global__ void __launch_bounds__(kSymThreads) sym_tile_kernel(const TL* __restrict__ tiles, int64_t n, int64_t nt,
                                                              const float* __restrict__ dcur, float* __restrict__ P) {
  __shared__ float dI[kSymTile], dJ[kSymTile];
  __shared__ float cpart[kSymThreads / 32][kSymTile];
  int64_t I, J;
  tile_coords(blockIdx.x, nt, I, J);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < kSymTile) {
    const int64_t i = I * kSymTile + threadIdx.x, j = J * kSymTile + threadIdx.x;
    dI[threadIdx.x] = i < n ? dcur[i] : 0.0f;
    dJ[threadIdx.x] = j < n ? dcur[j] : 0.0f;
  }
  const TL* T = tiles + static_cast<int64_t>(blockIdx.x) * kSymTile * kSymTile;
  const int r0 = warp * 16;
  float v[16][4];
#pragma unroll
  for (int rr = 0; rr < 16; ++rr) sym_load4(T + (r0 + rr) * kSymTile + 4 * lane, v[rr]);  // loads first
  __syncthreads();
  float xj[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) xj[k] = dJ[4 * lane + k];
  float rp[16], cacc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int rr = 0; rr < 16; ++rr) {
    const float xi = dI[r0 + rr];
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      s = fmaf(v[rr][k], xj[k], s);
      cacc[k] = fmaf(v[rr][k], xi, cacc[k]);
    }
    rp[rr] = s;
  }
  const float tot = SymTR<16, 16>::run(rp, lane);
  if ((lane & 1) == 0) P[(I * nt + J) * kSymTile + r0 + symtr_row(lane)] = tot;
  if (I != J) {
#pragma unroll
    for (int k = 0; k < 4; ++k) cpart[warp][4 * lane + k] = cacc[k];
    __syncthreads();
    if (threadIdx.x < kSymTile) {
      float s = 0.0f;
#pragma unroll
      for (int w = 0; w < kSymThreads / 32; ++w) s += cpart[w][threadIdx.x];
      P[(J * nt + I) * kSymTile + threadIdx.x] = s;
    }
  }
}

__device__ __forceinline__ void block_max2(unsigned long long a, unsigned long long b, unsigned long long* out) {
  __shared__ unsigned long long sa[32], sb[32];
  a = warp_max_u64(a);
  b = warp_max_u64(b);
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long ma = 0, mb = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
      ma = sa[w] > ma ? sa[w] : ma;
      mb = sb[w] > mb ? sb[w] : mb;
    }
    if (ma) atomicMax(out, ma);
    if (mb) atomicMax(out + 1, mb);
  }
}

// delta_new_i = c1_i - f_i * (sum of row i's nt slots, in slot order); the FP64 candidate x + delta_new; the
// maxima of |delta_new - delta| and |delta_new| into stats[0], stats[1].
__global__ void sym_finish_kernel(int64_t n, int64_t nt, const float* __restrict__ P, const float* __restrict__ c1,
                                  const float* __restrict__ rowfac, const float* __restrict__ dcur,
                                  float* __restrict__ dnew, const double* __restrict__ xc, double* __restrict__ xalt,
                                  unsigned long long* stats) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  unsigned long long chg = 0, mag = 0;
  if (i < n) {
    const int64_t I = i / kSymTile, rr = i % kSymTile;
    const float* p = P + I * nt * kSymTile + rr;
    float y = 0.0f;
    for (int64_t k = 0; k < nt; ++k) y += __ldcg(p + k * kSymTile);
    const float v = fmaf(-rowfac[i], y, c1[i]);
    chg = abs_bits(v - dcur[i]);
    mag = abs_bits(v);
    dnew[i] = v;
    xalt[i] = xc[i] + static_cast<double>(v);
  }
  block_max2(chg, mag, stats);
}

// Residual of x: r_i = b_i - sum_j a_ij x_j in FP64 (x == NULL: the zero vector, r = b), the inner
// right-hand side c1_i = fl32(r_i / a_ii) and the first inner iterate d1 = c1; max |r_i| and max |c1_i|
// into stats[0], stats[1].  Four rows per warp, two 16-byte column pairs per lane and row in flight.
__global__ void __launch_bounds__(256) sym_resid_kernel(int64_t n, const double* __restrict__ A, int64_t lda,
                                                        const double* __restrict__ x, const double* __restrict__ b,
                                                        const double* __restrict__ rinv, float* __restrict__ c1,
                                                        float* __restrict__ d1, unsigned long long* stats) {
  constexpr int R = 4;
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  unsigned long long mr = 0, mc = 0;
  for (int64_t i0 = (static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * R; i0 < n;
       i0 += warps * R) {
    double acc[R] = {0.0, 0.0, 0.0, 0.0};
    if (x) {
      const int rows = static_cast<int>(i64min(R, n - i0));
      int64_t j = 2 * lane;
      for (; j + 65 < n; j += 128) {
        const double2 x0 = __ldg(reinterpret_cast<const double2*>(x + j));
        const double2 x1 = __ldg(reinterpret_cast<const double2*>(x + j + 64));
        double2 a0[R], a1[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r < rows) {
            a0[r] = __ldcs(reinterpret_cast<const double2*>(A + (i0 + r) * lda + j));
            a1[r] = __ldcs(reinterpret_cast<const double2*>(A + (i0 + r) * lda + j + 64));
          }
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r < rows) {
            acc[r] = fma(a0[r].x, x0.x, acc[r]);
            acc[r] = fma(a0[r].y, x0.y, acc[r]);
            acc[r] = fma(a1[r].x, x1.x, acc[r]);
            acc[r] = fma(a1[r].y, x1.y, acc[r]);
          }
      }
      for (; j < n; j += 64)
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r < rows) {
            acc[r] = fma(A[(i0 + r) * lda + j], x[j], acc[r]);
            if (j + 1 < n) acc[r] = fma(A[(i0 + r) * lda + j + 1], x[j + 1], acc[r]);
          }
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = warp_sum(acc[r]);
    }
    if (lane < R && i0 + lane < n) {
      const int64_t i = i0 + lane;
      double dot = acc[0];
#pragma unroll
      for (int r = 1; r < R; ++r)
        if (lane == r) dot = acc[r];
      const double r = b[i] - dot;
      const float c = static_cast<float>(r * rinv[i]);
      c1[i] = c;
      d1[i] = c;
      const unsigned long long br = abs_bits(r), bc = abs_bits(c);
      mr = br > mr ? br : mr;
      mc = bc > mc ? bc : mc;
    }
  }
  block_max2(mr, mc, stats);
}

}  // namespace

int64_t sym_tiles_per_side(int64_t n) { return (n + kSymTile - 1) / kSymTile; }
int64_t sym_tile_count(int64_t n) {
  const int64_t nt = sym_tiles_per_side(n);
  return nt * (nt + 1) / 2;
}

cudaError_t launch_sym_pack(Narrow kind, const double* A, int64_t lda, int64_t n, const double* rinv, void* tiles,
                            float* rowfac, cudaStream_t s) {
  const int64_t nt = sym_tiles_per_side(n), count = sym_tile_count(n);
  if (kind == Narrow::F32)
    sym_pack_kernel<float><<<static_cast<unsigned>(count), 256, 0, s>>>(A, lda, n, nt, rinv, static_cast<float*>(tiles),
                                                                        rowfac);
  else
    sym_pack_kernel<__nv_bfloat16><<<static_cast<unsigned>(count), 256, 0, s>>>(
        A, lda, n, nt, rinv, static_cast<__nv_bfloat16*>(tiles), rowfac);
  return cudaGetLastError();
}

cudaError_t launch_sym_sweep(Narrow kind, const void* tiles, int64_t n, const float* dcur, float* P, const float* c1,
                             const float* rowfac, float* dnew, const double* xc, double* xalt, unsigned long long* stats,
                             cudaStream_t s) {
  const int64_t nt = sym_tiles_per_side(n), count = sym_tile_count(n);
  if (kind == Narrow::F32)
    sym_tile_kernel<float><<<static_cast<unsigned>(count), kSymThreads, 0, s>>>(static_cast<const float*>(tiles), n, nt,
                                                                              dcur, P);
  else
    sym_tile_kernel<__nv_bfloat16><<<static_cast<unsigned>(count), kSymThreads, 0, s>>>(
        static_cast<const __nv_bfloat16*>(tiles), n, nt, dcur, P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sym_finish_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(n, nt, P, c1, rowfac, dcur, dnew, xc, xalt,
                                                                          stats);
  return cudaGetLastError();
}

cudaError_t launch_sym_resid(int64_t n, const double* A, int64_t lda, const double* x, const double* b,
                             const double* rinv, float* c1, float* d1, unsigned long long* stats, cudaStream_t s) {
  int64_t blocks = (n + 31) / 32;  // 8 warps of 4 rows
  if (blocks > 152 * 16) blocks = 152 * 16;
  sym_resid_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(n, A, lda, x, b, rinv, c1, d1, stats);
  return cudaGetLastError();
}

}  // namespace jac
