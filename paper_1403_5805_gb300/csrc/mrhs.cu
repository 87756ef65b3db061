// Many right-hand sides: X (n x r) <- T X + C is a dense matrix-matrix product, so the sweep runs on
// the 5th-generation tensor cores.
//
// mrhs_sweep_kernel   one inner sweep of the mixed-precision refinement for r right-hand sides,
//                     delta^(m) = C1 - diag(1/a_ii) (N delta^(m-1)), on tcgen05: N (the BF16 copy of the
//                     off-diagonal part of A, the A operand) and delta (BF16, the B operand) are loaded by
//                     TMA into a 128-byte-swizzled shared-memory ring, one thread issues
//                     tcgen05.mma.kind::f16 (BF16 x BF16 -> FP32, M = 128, N = r, K = 16) into a tensor-
//                     memory accumulator, and four epilogue warps read it back with tcgen05.ld and apply
//                     the update, the FP64 candidate X + delta and the convergence reduction.
// mrhs_dense_kernel   the FP64 pass over A for all r columns on CUDA cores (shared-memory tiles, FP64
//                     FMA): either the residual R = B - A X (mixed path) or a plain FP64 Jacobi sweep
//                     X^(k) = D^-1 (B - (A - D) X^(k-1)) (FP64 path), Section 2.
//
// Vectors of r columns are stored column by column with a padded leading dimension ld: v[c*ld + i].
#include <cuda.h>

#include <cstdio>
#include <cstring>

#include "device_util.cuh"
#include "mrhs.cuh"
#include "tcgen05.cuh"
#include "splitfloat.cuh"

namespace jac {
namespace {

constexpr int kMTile = 128;                 // rows per tile (tcgen05 M)
constexpr int kMStages = 6;                 // ring depth of the widest blocks (r > 64)
// Up to 64 right-hand sides a 4-stage ring (97 KB) lets two CTAs share an SM, so the 256 row tiles of
// n = 32768 are all resident in one wave instead of 1.7 waves of one CTA per SM.
template <int R>
struct SweepCfg {
  static constexpr int kStages = R <= 64 ? 4 : kMStages;
  static constexpr int kCtasPerSm = R <= 64 ? 2 : 1;
};
constexpr int kSweepThreads = 192;          // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr int kATileBytes = kMTile * kKBlock * 2;  // 16 KB

struct SweepSmem {
  uint64_t full[kMStages];
  uint64_t empty[kMStages];
  uint64_t accum;
  uint32_t tmem;
  volatile int abort;
};

template <int R>
__global__ void __launch_bounds__(kSweepThreads, SweepCfg<R>::kCtasPerSm)
    mrhs_sweep_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      MrhsSweepParams p) {
  constexpr int kBTileBytes = R * kKBlock * 2;
  constexpr int kStageBytes = kATileBytes + kBTileBytes;
  constexpr uint32_t kTmemCols = R < 32 ? 32 : R;
  constexpr int kStages = SweepCfg<R>::kStages;
  extern __shared__ __align__(1024) unsigned char msmem[];
  __shared__ SweepSmem S;
  unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(msmem) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * kMTile;
  const int kb_count = static_cast<int>((p.n + kKBlock - 1) / kKBlock);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.accum, 1);
    S.abort = 0;
    mbar_init_fence();
  }
  if (warp == 1) tmem_alloc(&S.tmem, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;

  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < kb_count; ++kb) {
        const int s = kb % kStages;
        const uint32_t par = ((kb / kStages) & 1) ^ 1;
        if (S.abort || !mbar_wait(&S.empty[s], par) || S.abort) {
          S.abort = 1;
          atomicCAS(p.status, 0, kStatusTimeout);
          break;
        }
        unsigned char* a = ring + s * kStageBytes;
        mbar_arrive_expect_tx(&S.full[s], kStageBytes);
        tma_load_2d(a, &tmA, kb * kKBlock, static_cast<int>(m0), &S.full[s]);
        tma_load_2d(a + kATileBytes, &tmB, kb * kKBlock, 0, &S.full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = mma_idesc(kMTile, R);
      for (int kb = 0; kb < kb_count; ++kb) {
        const int s = kb % kStages;
        if (S.abort || !mbar_wait(&S.full[s], (kb / kStages) & 1)) {
          S.abort = 1;
          atomicCAS(p.status, 0, kStatusTimeout);
          break;
        }
        tc_fence_after();
        const uint32_t a = cvta_smem(ring + s * kStageBytes);
        const uint32_t b = a + kATileBytes;
#pragma unroll
        for (int k = 0; k < kKBlock / 16; ++k)  // K = 16 BF16 = 32 bytes per instruction
          mma_bf16(tmem, sw128_desc(a + 32 * k), sw128_desc(b + 32 * k), idesc, (kb | k) != 0);
        mma_commit(&S.empty[s]);  // the stage is free once these MMAs have read it
      }
      mma_commit(&S.accum);  // the accumulator is complete once every MMA has finished
    }
  } else {
    // epilogue warps 2..5: warp w reads TMEM lanes 32*(w % 4) .. +31 (one output row per thread)
    const int q = warp & 3;
    const int64_t i = m0 + 32 * q + lane;
    bool ok = mbar_wait(&S.accum, 0) && !S.abort;
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;  // tcgen05.ld below is warp-collective
    tc_fence_after();
    unsigned long long mchg = 0, mmag = 0;
    if (ok) {
      const float f = i < p.n ? p.rowfac[i] : 0.0f;
#pragma unroll 1
      for (int c0 = 0; c0 < R; c0 += 32) {
        float acc[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(c0), acc);
        if (i < p.n) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (c0 + j >= R) break;
            const int64_t o = static_cast<int64_t>(c0 + j) * p.ld + i;
            const float v = fmaf(-f, acc[j], p.c1[o]);
            const float old = p.dc[o];
            p.dn[o] = v;
            p.dnh[o] = __float2bfloat16_rn(v);
            p.xalt[o] = p.xc[o] + static_cast<double>(v);
            const unsigned long long a1 = abs_bits(v - old), a2 = abs_bits(v);
            mchg = a1 > mchg ? a1 : mchg;
            mmag = a2 > mmag ? a2 : mmag;
          }
        }
      }
    } else {
      atomicCAS(p.status, 0, kStatusTimeout);
    }
    mchg = warp_max_u64(mchg);
    mmag = warp_max_u64(mmag);
    if (lane == 0) {
      if (mchg) atomicMax(p.stats + 0, mchg);
      if (mmag) atomicMax(p.stats + 1, mmag);
    }
  }
  // every MMA has been waited for (accum barrier) or none is in flight (abort); free TMEM
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ---------------------------------------------------------------- FP64 dense pass, all r columns
constexpr int kDM = 64;   // rows per tile
constexpr int kDN = 64;   // columns (right-hand sides) per tile
constexpr int kDK = 32;   // K step
constexpr int kDThreads = 256;

// Column worked on by tile column c (c < nact).
__device__ __forceinline__ int col_of(const MrhsDenseParams& p, int c) { return p.cols ? __ldg(p.cols + c) : c; }

// FP64 dense pass tiles: 32 rows x 64 columns per block, so that the 1024 row tiles of n = 32768 spread
// over the SMs within a few percent (64-row tiles left a quarter of the SMs with 4 blocks and the rest
// with 3, and the FP64 pipes of the busier SMs set the time).
constexpr int kFM = kMrhsDenseRows;
constexpr int kFN = 64;
constexpr int kFK = 32;

// mode 0: residual R = B - A X; writes C1 = R / a_ii (FP32), delta^(1) = C1 (FP32 + BF16), and the
//         per-column max |R|.
// mode 1: FP64 Jacobi sweep X^(k) = (B - A X + a_ii x_i) / a_ii; writes X^(k) and the max |change|.
__global__ void __launch_bounds__(kDThreads) mrhs_dense_kernel(MrhsDenseParams p) {
  __shared__ double As[kFK][kFM + 1];
  __shared__ double Xs[kFK][kFN + 1];
  const int tid = threadIdx.x;
  const int tr = tid / 32, tc = tid % 32;  // 8 x 32 threads, each 4 rows (tr + 8u) x 2 columns (tc + 32v)
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * kFM;
  const int c0 = blockIdx.y * kFN;
  double acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = 0.0;
  for (int64_t k0 = 0; k0 < p.n; k0 += kFK) {
    // A tile: kFM rows x kFK columns (row-major A), stored transposed As[k][m]
    for (int e = tid; e < kFM * kFK; e += kDThreads) {
      const int m = e / kFK, k = e % kFK;
      const int64_t gi = m0 + m, gk = k0 + k;
      As[k][m] = (gi < p.n && gk < p.n) ? __ldg(p.A + gi * p.lda + gk) : 0.0;
    }
    // X tile: kFK rows x kFN columns from the column-major X (x[c*ld + k])
    for (int e = tid; e < kFK * kFN; e += kDThreads) {
      const int c = e / kFK, k = e % kFK;
      const int64_t gk = k0 + k;
      Xs[k][c] = (gk < p.n && c0 + c < p.nact) ? p.x[static_cast<int64_t>(col_of(p, c0 + c)) * p.ld + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kFK; ++k) {
      double a[4], x[2];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[k][tr + 8 * u];
#pragma unroll
      for (int v = 0; v < 2; ++v) x[v] = Xs[k][tc + 32 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) acc[u][v] = fma(a[u], x[v], acc[u][v]);
    }
    __syncthreads();
  }
  unsigned long long mloc[2] = {0, 0};
  double sq[2] = {0.0, 0.0};
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = m0 + tr + 8 * u;
    if (i >= p.n) continue;
    const double di = p.d[i], ri = p.rinv[i];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      if (c0 + tc + 32 * v >= p.nact) continue;
      const int c = col_of(p, c0 + tc + 32 * v);
      const int64_t o = static_cast<int64_t>(c) * p.ld + i;
      const double b = p.b[o];
      if (p.mode == 0) {
        const double r = b - acc[u][v];
        const float cc = static_cast<float>(r * ri);
        p.c1[o] = cc;
        p.d1[o] = cc;
        p.d1h[o] = __float2bfloat16_rn(cc);
        const unsigned long long bits = abs_bits(r);
        mloc[v] = bits > mloc[v] ? bits : mloc[v];
      } else {
        const double xo = p.x[o];
        const double s = fma(-di, xo, acc[u][v]);
        const double xi = (b - s) * ri;
        p.xn[o] = xi;
        const unsigned long long bits = abs_bits(p.resid_norm ? di * (xi - xo) : xi - xo);
        mloc[v] = bits > mloc[v] ? bits : mloc[v];
        sq[v] = fma(xi - xo, xi - xo, sq[v]);  // rows in the order u = 0..3
      }
    }
  }
  if (p.colsq) {
    // the tile's 8 row groups summed per column in a fixed order (As is free after the last K step)
    double* part = &As[0][0];  // [8][kFN + 1]
#pragma unroll
    for (int v = 0; v < 2; ++v) part[tr * (kFN + 1) + tc + 32 * v] = sq[v];
    __syncthreads();
    if (tid < kFN && c0 + tid < p.nact) {
      double t = 0.0;
      for (int g = 0; g < 8; ++g) t += part[g * (kFN + 1) + tid];
      p.colsq[static_cast<int64_t>(blockIdx.x) * p.r + col_of(p, c0 + tid)] = t;
    }
  }
#pragma unroll
  for (int v = 0; v < 2; ++v)
    if (c0 + tc + 32 * v < p.nact && mloc[v]) atomicMax(p.colmax + col_of(p, c0 + tc + 32 * v), mloc[v]);
}

// ------------------------------------------------- split-float residual pass (FP32 units), all r columns
// R = B - A X with the split-float arithmetic of splitfloat.cuh: tiles of A are split (row scale 2^-e_i)
// as they are staged into shared memory, X arrives as two FP32 words per entry (column scale 2^-g_c),
// and every product is accumulated float-float.  The tile schedule is the FP64 pass's: 64 rows x 16 NC
// columns per CTA, each thread 4 rows x NC columns.  Writes what mode 0 of the FP64 pass writes.
template <int NC>
__global__ void __launch_bounds__(kDThreads, 2) mrhs_split_resid_kernel(MrhsDenseParams p) {
  constexpr int kN = 16 * NC;
  __shared__ float2 As[kDK][kDM + 1];  // (hi, lo) of the split A tile, transposed
  __shared__ float2 Xs[kDK][kN + 1];   // (hi, lo) of the X tile
  __shared__ int sh_row[kDM], g_col[kN];
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * kDM;
  const int c0 = blockIdx.y * kN;
  if (tid < kDM) sh_row[tid] = m0 + tid < p.n ? p.rexp[m0 + tid] : 0;
  if (tid < kN) g_col[tid] = c0 + tid < p.nact ? p.xexp[col_of(p, c0 + tid)] : 0;
  __syncthreads();
  FF acc[4][NC];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < NC; ++b) acc[a][b] = FF{0.0f, 0.0f};
  for (int64_t k0 = 0; k0 < p.n; k0 += kDK) {
    for (int e = tid; e < kDM * kDK; e += kDThreads) {
      const int m = e / kDK, k = e % kDK;
      const int64_t gi = m0 + m, gk = k0 + k;
      const double a = (gi < p.n && gk < p.n) ? __ldg(p.A + gi * p.lda + gk) : 0.0;
      float hi, lo;
      split_scaled(a, sh_row[m], hi, lo);
      As[k][m] = make_float2(hi, lo);
    }
    for (int e = tid; e < kDK * kN; e += kDThreads) {
      const int c = e / kDK, k = e % kDK;
      const int64_t gk = k0 + k;
      const float2 v = (gk < p.n && c0 + c < p.nact) ? __ldg(p.xs + static_cast<int64_t>(col_of(p, c0 + c)) * p.ld + gk)
                                                    : make_float2(0.0f, 0.0f);
      Xs[k][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kDK; ++k) {
      float2 a[4], x[NC];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[k][tr + 16 * u];
#pragma unroll
      for (int v = 0; v < NC; ++v) x[v] = Xs[k][tc + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < NC; ++v) ff_fma(acc[u][v], a[u].x, a[u].y, x[v].x, x[v].y);
      if ((k & 7) == 7) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < NC; ++v) ff_renorm(acc[u][v]);
      }
    }
    __syncthreads();
  }
  unsigned long long mloc[NC];
#pragma unroll
  for (int v = 0; v < NC; ++v) mloc[v] = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = m0 + tr + 16 * u;
    if (i >= p.n) continue;
    const double ri = p.rinv[i];
    const double si = pow2(sh_row[tr + 16 * u]);
#pragma unroll
    for (int v = 0; v < NC; ++v) {
      if (c0 + tc + 16 * v >= p.nact) continue;
      const int c = col_of(p, c0 + tc + 16 * v);
      const int64_t o = static_cast<int64_t>(c) * p.ld + i;
      const double dot =
          (static_cast<double>(acc[u][v].hi) + static_cast<double>(acc[u][v].lo)) * si * pow2(g_col[tc + 16 * v]);
      const double r = p.b[o] - dot;
      const float cc = static_cast<float>(r * ri);
      p.c1[o] = cc;
      p.d1[o] = cc;
      p.d1h[o] = __float2bfloat16_rn(cc);
      const unsigned long long bits = abs_bits(r);
      mloc[v] = bits > mloc[v] ? bits : mloc[v];
    }
  }
#pragma unroll
  for (int v = 0; v < NC; ++v)
    if (c0 + tc + 16 * v < p.nact && mloc[v]) atomicMax(p.colmax + col_of(p, c0 + tc + 16 * v), mloc[v]);
}

// One CTA per column: g_c = split exponent of max_i |x_ic|, then xs = the two FP32 words of x 2^-g_c.
__global__ void mrhs_split_x_kernel(int64_t n, int64_t ld, const double* __restrict__ x, float2* __restrict__ xs,
                                    int* __restrict__ xexp) {
  __shared__ unsigned long long sh[32];
  const int64_t c = blockIdx.x;
  const double* col = x + c * ld;
  unsigned long long m = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned long long b = abs_bits(col[i]);
    m = b > m ? b : m;
  }
  m = warp_max_u64(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  unsigned long long t = 0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t = sh[w] > t ? sh[w] : t;
  const int g = split_exponent(t);
  if (threadIdx.x == 0) xexp[c] = g;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xs[c * ld + i] = split_x(col[i], g);
}

template <int R>
cudaError_t launch_sweep_r(const CUtensorMap& ta, const CUtensorMap& tb, const MrhsSweepParams& p, cudaStream_t s) {
  constexpr int smem = SweepCfg<R>::kStages * (kATileBytes + R * kKBlock * 2) + 1024;
  cudaError_t e = cudaFuncSetAttribute(mrhs_sweep_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = static_cast<unsigned>((p.n + kMTile - 1) / kMTile);
  mrhs_sweep_kernel<R><<<grid, kSweepThreads, smem, s>>>(ta, tb, p);
  return cudaGetLastError();
}

__global__ void mrhs_init_kernel(int64_t n, int64_t r, int64_t ld, const double* __restrict__ b,
                                 const double* __restrict__ rinv, float* c1, float* d1, __nv_bfloat16* d1h,
                                 unsigned long long* colmax) {
  const int64_t total = n * r;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = e / n, i = e % n;
    const int64_t o = c * ld + i;
    const double v = b[o];
    const float cc = static_cast<float>(v * rinv[i]);
    c1[o] = cc;
    d1[o] = cc;
    d1h[o] = __float2bfloat16_rn(cc);
    atomicMax(colmax + c, abs_bits(v));
  }
}

}  // namespace

cudaError_t launch_mrhs_init(int64_t n, int64_t r, int64_t ld, const double* b, const double* rinv, float* c1,
                             float* d1, __nv_bfloat16* d1h, unsigned long long* colmax, cudaStream_t s) {
  int64_t blocks = (n * r + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  mrhs_init_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(n, r, ld, b, rinv, c1, d1, d1h, colmax);
  return cudaGetLastError();
}

bool mrhs_supported_r(int64_t r) { return r == 16 || r == 32 || r == 64 || r == 128; }

cudaError_t launch_mrhs_sweep(const void* Nlow, const void* dh, const MrhsSweepParams& p, cudaStream_t s) {
  CUtensorMap ta, tb;
  if (!make_map(&ta, Nlow, p.n, p.n, p.ld, kMTile)) return cudaErrorInvalidValue;
  if (!make_map(&tb, dh, p.n, p.r, p.ld, static_cast<int>(p.r))) return cudaErrorInvalidValue;
  switch (p.r) {
    case 16: return launch_sweep_r<16>(ta, tb, p, s);
    case 32: return launch_sweep_r<32>(ta, tb, p, s);
    case 64: return launch_sweep_r<64>(ta, tb, p, s);
    case 128: return launch_sweep_r<128>(ta, tb, p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_mrhs_dense(const MrhsDenseParams& p, cudaStream_t s) {
  if (p.nact < 1) return cudaSuccess;
  if (p.xs && p.mode == 0) {
    const int nc = p.nact <= 16 ? 1 : (p.nact <= 32 ? 2 : 4);
    const dim3 grid(static_cast<unsigned>((p.n + kDM - 1) / kDM),
                    static_cast<unsigned>((p.nact + 16 * nc - 1) / (16 * nc)));
    if (nc == 1)
      mrhs_split_resid_kernel<1><<<grid, kDThreads, 0, s>>>(p);
    else if (nc == 2)
      mrhs_split_resid_kernel<2><<<grid, kDThreads, 0, s>>>(p);
    else
      mrhs_split_resid_kernel<4><<<grid, kDThreads, 0, s>>>(p);
    return cudaGetLastError();
  }
  const dim3 grid(static_cast<unsigned>((p.n + kFM - 1) / kFM), static_cast<unsigned>((p.nact + kFN - 1) / kFN));
  mrhs_dense_kernel<<<grid, kDThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_mrhs_split_x(int64_t n, int64_t r, int64_t ld, const double* x, float2* xs, int* xexp,
                                cudaStream_t s) {
  mrhs_split_x_kernel<<<static_cast<unsigned>(r), 256, 0, s>>>(n, ld, x, xs, xexp);
  return cudaGetLastError();
}

}  // namespace jac
