// FP64-accurate residual R = B - A X for many right-hand sides on the tcgen05 tensor cores, by splitting
// A and X into BF16 "digits" whose products the tensor cores add up exactly (the error-free splitting
// of Ozaki, Ogita, Oishi & Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Splitting.  Row i of the off-diagonal part of A is scaled by 2^-(e_i + 1), e_i the exponent with
// max_{j != i} |a_ij| < 2^e_i, so every scaled entry t lies in (-1/2, 1/2).  t is rounded to a signed
// fixed-point integer T = round(t 2^56) (|T| <= 2^55) and written in balanced base 256,
//     T = sum_{p=1..7} d_p 256^(7-p),   d_2 .. d_7 in [-128, 127],   |d_1| <= 128,
// so a_ij = 2^(e_i + 1) (sum_p d_p 2^-8p + r_ij) with |r_ij| <= 2^-57.  Each column c of X is split the
// same way with its own exponent g_c (max_i |x_ic| < 2^g_c) into digits f_q.  Digits are stored as BF16
// values d_p 2^-8(p-1) (any integer of at most 8 significant bits times a power of two is exact in BF16).
//
// Products.  a_ij x_jc = 2^(e_i + g_c + 2 - 16) sum_{p,q} (d_p 2^-8(p-1)) (f_q 2^-8(q-1)).  Pairs with
// p + q <= 8 are kept; the dropped ones (p + q >= 9) are below 2^-56 of the leading product's scale, and
// the representation errors r_ij below 2^-57 of the row and column maxima.  The tensor cores multiply one
// BF16 digit matrix of A (M = 128 rows x K) by several BF16 digit blocks of X (N = digits x columns) into
// FP32 accumulators in tensor memory.  Every digit product is an integer times 2^-8(p+q-2) of magnitude at
// most 128 * 128 = 2^14 in those units, so a sum of 1024 of them is at most 2^24 and exact in FP32
// whatever the order of the additions: the accumulator is read out every 1024 columns of K (one chunk)
// and its exact chunk sums are added into a float-float (two FP32 words) accumulator per output entry
// with Knuth's two-sum, lowest digit levels first.  The diagonal term a_ii x_ic is applied in FP64.
//
// Kernel.  One CTA per 128 rows and RC columns of X (and, when the row tiles alone would leave part of
// the last wave of CTAs idle, per part of the K range: the parts' float-float sums go to scratch and a
// second launch adds them in part order): warp 0 issues the TMA loads (the A digit tile, 128 x 64 BF16,
// and one X digit block of RC x 64 per digit) into a 128-byte-swizzled ring of up to 4 stages; one
// thread of warp 1 issues tcgen05.mma.kind::f16 (M = 128, N = digits x RC, at most 256 per instruction,
// K = 16) into tensor memory; the readout warps read a finished chunk with tcgen05.ld, add it into their
// registers (one output row per thread) and hand the columns back.  For RC <= 32 a group's accumulator
// fits in 256 columns and two such buffers alternate per chunk, so the readout of one chunk overlaps
// the products of the next; for RC = 64 (up to 448 columns) one buffer serves.  The groups run from A
// digit 7 (one X digit, the lowest level) to A digit 1 (seven X digits).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "device_util.cuh"
#include "mrhs.cuh"
#include "splitfloat.cuh"
#include "tcgen05.cuh"

namespace jac {
namespace {

constexpr int kOzTile = 128;              // rows per CTA (tcgen05 M)
constexpr int kOzChunkKB = 16;            // 64-column K blocks per exact FP32 chunk: 1024 columns
constexpr int kOzBufCols = 256;           // tensor-memory columns per accumulator buffer
constexpr int kOzTmemCols = 2 * kOzBufCols;
constexpr int kOzATile = kOzTile * kKBlock * 2;  // 16 KB
constexpr int kExpNonfinite = 0x7FFFFFFF;        // exponent marker of a row or column holding inf / NaN

// Exponent e with m < 2^e for the maximum m whose high word (sign cleared) is hb; 0 for m = 0 and the
// non-finite marker for inf / NaN.
__device__ __forceinline__ int oz_exponent(uint32_t hb) {
  const int be = static_cast<int>(hb >> 20);
  if (be == 0x7FF) return kExpNonfinite;
  if (hb == 0) return 0;  // zero, or a maximum below 2^-1042: its digits are all zero below
  return be == 0 ? -1022 : be - 1022;
}

// The 7 balanced base-256 digits of v 2^-(e + 1) (|v| < 2^e), most significant first.
__device__ __forceinline__ void oz_digits(double v, int e, int (&d)[kOzDigits]) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(v));
  const int eb = static_cast<int>((bits >> 52) & 0x7FFu);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  int eu = -1022;
  if (eb != 0) {
    m |= 1ull << 52;
    eu = eb - 1023;
  }
  // v 2^-(e+1) 2^56 = m 2^(eu - 52 - e - 1 + 56): shift m by sh (sh <= 2 since |v| < 2^e)
  const int sh = eu - e + 3;
  long long T;
  if (m == 0 || e == kExpNonfinite) {
    T = 0;
  } else if (sh >= 0) {
    T = static_cast<long long>(m << sh);
  } else {
    const int k = -sh;
    T = k >= 60 ? 0 : static_cast<long long>((m + (1ull << (k - 1))) >> k);  // round half up
  }
  if (bits >> 63) T = -T;
#pragma unroll
  for (int p = kOzDigits - 1; p >= 1; --p) {
    const int dd = static_cast<int>((T + 128) & 255) - 128;
    d[p] = dd;
    T = (T - dd) >> 8;  // exact: T - dd is a multiple of 256
  }
  d[0] = static_cast<int>(T);  // |d_1| <= 128
}

__device__ __forceinline__ __nv_bfloat16 oz_digit_value(int d, int p) {
  // d 2^-8p for the digit of index p (0-based): exact in FP32 and BF16
  return __float2bfloat16_rn(__int2float_rn(d) * __uint_as_float(static_cast<uint32_t>(127 - 8 * p) << 23));
}

// One warp per row (grid-stride over the nr padded rows): e_i from the off-diagonal maximum, then the
// digits of every entry, two columns per lane and step (BF16 pairs), zero on the diagonal, in the column
// padding [n, ld) and in the rows [n, nr).
__global__ void oz_split_a_kernel(const double* __restrict__ A, int64_t lda, int64_t n, int64_t nr, int64_t ld,
                                  __nv_bfloat16* __restrict__ dig, int* __restrict__ aexp) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t plane = nr * ld;  // elements per digit matrix
  for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nr; i += static_cast<int64_t>(gridDim.x) * wpb) {
    const double* Ai = A + i * lda;
    uint32_t mb = 0;
    if (i < n)
      for (int64_t j = lane; j < n; j += 32)
        if (j != i) mb = max(mb, abs_hi(Ai[j]));
    mb = __reduce_max_sync(0xffffffffu, mb);
    const int e = oz_exponent(mb);
    if (lane == 0 && i < n) aexp[i] = e;
    for (int64_t j = 2 * lane; j < ld; j += 64) {
      double v0 = 0.0, v1 = 0.0;
      if (i < n) {
        if (j + 1 < n) {
          const double2 v = *reinterpret_cast<const double2*>(Ai + j);  // rows are 16-byte aligned, j even
          v0 = v.x;
          v1 = v.y;
        } else if (j < n) {
          v0 = Ai[j];
        }
        if (j == i) v0 = 0.0;
        if (j + 1 == i) v1 = 0.0;
      }
      int d0[kOzDigits], d1[kOzDigits];
      oz_digits(v0, e, d0);
      oz_digits(v1, e, d1);
#pragma unroll
      for (int p = 0; p < kOzDigits; ++p) {
        __nv_bfloat162 w;
        w.x = oz_digit_value(d0[p], p);
        w.y = oz_digit_value(d1[p], p);
        *reinterpret_cast<__nv_bfloat162*>(dig + p * plane + i * ld + j) = w;
      }
    }
  }
}

// One CTA per column c of X (x[c*ld + i]): g_c from max_i |x_ic|, then the digits, stored q-major:
// digit q of column c at xd[(q*r + c)*ld + i]; entries i in [n, ld) are zero.
__global__ void oz_split_x_kernel(int64_t n, int64_t r, int64_t ld, const double* __restrict__ x,
                                  __nv_bfloat16* __restrict__ xd, int* __restrict__ xexp) {
  __shared__ uint32_t sh[32];
  const int64_t c = blockIdx.x;
  const double* col = x + c * ld;
  uint32_t m = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = max(m, abs_hi(col[i]));
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  uint32_t t = 0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t = max(t, sh[w]);
  const int g = oz_exponent(t);
  if (threadIdx.x == 0) xexp[c] = g;
  for (int64_t i = threadIdx.x; i < ld; i += blockDim.x) {
    int d[kOzDigits];
    oz_digits(i < n ? col[i] : 0.0, g, d);
#pragma unroll
    for (int q = 0; q < kOzDigits; ++q) xd[(q * r + c) * ld + i] = oz_digit_value(d[q], q);
  }
}

// v 2^k for any k (several exact power-of-two factors; over- and underflow as the true product).
__device__ __forceinline__ double scale2(double v, int k) {
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int kk = k < -1000 ? -1000 : (k > 1000 ? 1000 : k);
    v *= pow2(kk);
    k -= kk;
  }
  return v;
}

__device__ __forceinline__ void ff_add(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// Per-CTA column count RC (16, 32 or 64 columns of X) fixes the geometry: the readout warps (one output
// row per thread and TMEM lane quadrant; with 64 columns two warps per quadrant, 32 columns each), the
// stage size (A digit tile + 7 X digit blocks of RC rows), the ring depth within 217 KB, and the tensor-
// memory accumulators: a group's nq * RC columns (at most 448) in one buffer for RC = 64, or two
// alternating 256-column buffers for RC <= 32 (so that the readout of one chunk overlaps the next).
template <int RC>
struct OzCfg {
  static constexpr int kReadWarps = RC == 64 ? 8 : 4;
  static constexpr int kThreads = 64 + 32 * kReadWarps;
  static constexpr int kXBlock = RC * kKBlock * 2;
  static constexpr int kStage = kOzATile + kOzDigits * kXBlock;
  static constexpr int kStages = (217 * 1024) / kStage < 4 ? (217 * 1024) / kStage : 4;
  static constexpr int kBufs = kOzDigits * RC <= kOzBufCols ? 2 : 1;
  static constexpr int kDigitsPerMma = kOzBufCols / RC < kOzDigits ? kOzBufCols / RC : kOzDigits;
  static constexpr int kColsPerWarp = RC == 64 ? 32 : RC;
  static constexpr int kSmem = kStages * kStage + 1024;
  static_assert(kStages >= 2, "ring needs two stages");
  static_assert(kOzDigits * RC <= kOzTmemCols, "a group's accumulator fits tensor memory");
};

struct OzSmem {
  uint64_t full[4];
  uint64_t empty[4];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t done;
  uint32_t tmem;
  volatile int abort;
  int active[64];  // columns of this CTA that are written (1) or skipped (retired columns)
};

// The residual of one tile: rows [m0, m0 + 128) and columns [c0, c0 + RC) of X, A's digits through the
// tensor map *tmA, X's digits through *tmX (kernel parameters or maps in global memory).
// Only the chunks [ch0, ch1) of K (1024 columns each) are summed; with nparts > 1 the tile's float-float sums
// go to the part scratch (part index part) for oz_finish_kernel, else the tile applies the epilogue itself.
template <int RC>
__device__ __forceinline__ void oz_resid_tile(const CUtensorMap* tmA_, const CUtensorMap* tmX_,
                                              const OzResidParams& p, int64_t m0, int c0, int ch0, int ch1,
                                              int nparts, int part) {
  using C = OzCfg<RC>;
  constexpr int S_ = C::kStages;
  constexpr int NB = C::kBufs;
  extern __shared__ __align__(1024) unsigned char osmem[];
  __shared__ OzSmem S;
  unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(osmem) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const CUtensorMap& tmA = *tmA_;
  const CUtensorMap& tmX = *tmX_;
  const int kb_count = static_cast<int>((p.n + kKBlock - 1) / kKBlock);
  const int kb_lo = ch0 * kOzChunkKB, kb_hi = min(kb_count, ch1 * kOzChunkKB);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S_; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.tfull[b], 1);
      mbar_init(&S.tempty[b], C::kReadWarps);  // one arrival per readout warp
    }
    mbar_init(&S.done, 1);
    S.abort = 0;
    mbar_init_fence();
  }
  if (threadIdx.x < RC) S.active[threadIdx.x] = p.cols ? 0 : 1;
  __syncthreads();
  if (p.cols && threadIdx.x == 0)
    for (int64_t k = 0; k < p.nact; ++k) {
      const int c = p.cols[k] - c0;
      if (c >= 0 && c < RC) S.active[c] = 1;
    }
  if (warp == 1) tmem_alloc(&S.tmem, kOzTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int gi = 0; gi < kOzDigits && !S.abort; ++gi) {
        const int pd = kOzDigits - 1 - gi;  // A digit (0-based); X digits 0 .. gi
        const int nq = gi + 1;
        for (int kb = kb_lo; kb < kb_hi; ++kb, ++it) {
          const int s = it % S_;
          if (S.abort || !mbar_wait(&S.empty[s], ((it / S_) & 1) ^ 1, p.wait_ns) || S.abort) {
            S.abort = 1;
            atomicCAS(p.status, 0, kStatusTimeout);
            break;
          }
          unsigned char* st = ring + s * C::kStage;
          mbar_arrive_expect_tx(&S.full[s], kOzATile + nq * C::kXBlock);
          tma_load_2d(st, &tmA, kb * kKBlock, static_cast<int>(pd * p.nr + m0), &S.full[s]);
          for (int q = 0; q < nq; ++q)
            tma_load_2d(st + kOzATile + q * C::kXBlock, &tmX, kb * kKBlock, static_cast<int>(q * p.r + c0),
                        &S.full[s]);
        }
      }
      // wait (bounded) for the copies still in flight before the CTA can exit
      for (int k = it - 1; k >= 0 && k >= it - S_; --k) mbar_wait(&S.full[k % S_], (k / S_) & 1, p.wait_ns);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, t = 0;
      for (int gi = 0; gi < kOzDigits && !S.abort; ++gi) {
        const int nq = gi + 1;
        for (int ch = ch0; ch < ch1 && !S.abort; ++ch, ++t) {
          const int b = t % NB, u = t / NB;
          if (!mbar_wait(&S.tempty[b], (u & 1) ^ 1, p.wait_ns) || S.abort) {
            S.abort = 1;
            atomicCAS(p.status, 0, kStatusTimeout);
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + static_cast<uint32_t>(b * kOzBufCols);
          const int kb1 = min(kb_count, (ch + 1) * kOzChunkKB);
          for (int kb = ch * kOzChunkKB; kb < kb1; ++kb, ++it) {
            const int s = it % S_;
            if (!mbar_wait(&S.full[s], (it / S_) & 1, p.wait_ns) || S.abort) {
              S.abort = 1;
              atomicCAS(p.status, 0, kStatusTimeout);
              break;
            }
            tc_fence_after();
            const uint32_t a = cvta_smem(ring + s * C::kStage);
            const uint32_t bx = a + kOzATile;
#pragma unroll
            for (int k = 0; k < kKBlock / 16; ++k) {
              const uint32_t accum = (kb != ch * kOzChunkKB || k != 0) ? 1u : 0u;
              // at most 256 accumulator columns per instruction: digits [q0, q0 + nd) of X
              for (int q0 = 0; q0 < nq; q0 += C::kDigitsPerMma) {
                const int nd = min(C::kDigitsPerMma, nq - q0);
                mma_bf16(acc + static_cast<uint32_t>(q0 * RC), sw128_desc(a + 32 * k),
                         sw128_desc(bx + q0 * C::kXBlock + 32 * k), mma_idesc(kOzTile, nd * RC), accum);
              }
            }
            mma_commit(&S.empty[s]);
          }
          mma_commit(&S.tfull[b]);
        }
      }
      // every MMA issued has completed once this commit arrives: only then may tensor memory be freed
      mma_commit(&S.done);
      mbar_wait(&S.done, 0, p.wait_ns);
    }
  } else {
    // readout warps: warp w owns tensor-memory lanes 32 (w % 4) .. + 31 (one output row per thread) and,
    // with 64 columns, the column half (w - 2) / 4
    constexpr int CW = C::kColsPerWarp;
    const int qd = warp & 3;
    const int cw = RC == 64 ? ((warp - 2) >> 2) * 32 : 0;  // first column of this warp
    const int64_t i = m0 + 32 * qd + lane;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * qd) << 16);
    float hi[CW], lo[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) hi[c] = lo[c] = 0.0f;
    bool ok = true;
    int t = 0;
    for (int gi = 0; gi < kOzDigits && ok; ++gi) {
      const int nq = gi + 1;
      for (int ch = ch0; ch < ch1 && ok; ++ch, ++t) {
        const int b = t % NB, u = t / NB;
        bool got = lane == 0 ? (mbar_wait(&S.tfull[b], u & 1, p.wait_ns) && !S.abort) : false;
        got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;  // tcgen05.ld is warp-collective
        if (!got) {
          ok = false;
          break;
        }
        tc_fence_after();
        // lowest level first: X digit nq-1 (level pd + nq) down to X digit 0
        for (int q = nq - 1; q >= 0; --q) {
          const uint32_t col = static_cast<uint32_t>(b * kOzBufCols + q * RC + cw);
          if constexpr (CW == 32) {
            float v[32];
            tmem_ld32(lane_base + col, v);
#pragma unroll
            for (int c = 0; c < 32; ++c) ff_add(hi[c], lo[c], v[c]);
          } else {
            float v[16];
            tmem_ld16(lane_base + col, v);
#pragma unroll
            for (int c = 0; c < 16; ++c) ff_add(hi[c], lo[c], v[c]);
          }
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) {  // renormalise: |lo| <= ulp(hi) / 2
          const float z = __fadd_rn(hi[c], lo[c]);
          lo[c] = __fsub_rn(lo[c], __fsub_rn(z, hi[c]));
          hi[c] = z;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.tempty[b]);
      }
    }
    if (!ok) {
      if (lane == 0) {
        S.abort = 1;
        atomicCAS(p.status, 0, kStatusTimeout);
      }
    } else if (nparts > 1) {
      // this part's sums of rows [m0, m0 + 128) and the warp's columns, for oz_finish_kernel
      if (i < p.n) {
#pragma unroll
        for (int c = 0; c < CW; ++c)
          p.part[(static_cast<int64_t>(part) * p.r + c0 + cw + c) * p.ld + i] = make_float2(hi[c], lo[c]);
      }
    } else {
      const bool row_ok = i < p.n;
      const int e = row_ok ? p.aexp[i] : 0;
      const double di = row_ok ? p.d[i] : 0.0, ri = row_ok ? p.rinv[i] : 0.0;
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        const int col = c0 + cw + c;
        const int64_t o = static_cast<int64_t>(col) * p.ld + i;
        unsigned long long bits = 0;
        if (row_ok && S.active[cw + c]) {
          const int g = p.xexp[col];
          double dot;
          if (e == kExpNonfinite || g == kExpNonfinite)
            dot = __longlong_as_double(0x7FF8000000000000ll);
          else
            dot = scale2(static_cast<double>(hi[c]) + static_cast<double>(lo[c]), e + g + 2 - 16);
          const double r = fma(-di, p.x[o], p.b[o]) - dot;
          const float cc = static_cast<float>(r * ri);
          p.c1[o] = cc;
          p.d1[o] = cc;
          if (p.d1h) p.d1h[o] = __float2bfloat16_rn(cc);
          bits = abs_bits(r);
        }
        if (S.active[cw + c]) {  // warp-uniform
          bits = warp_max_u64(bits);
          if (lane == 0 && bits) atomicMax(p.colmax + col, bits);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kOzTmemCols);
  }
}

template <int RC>
__global__ void __launch_bounds__(OzCfg<RC>::kThreads, 1)
    oz_resid_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
                    OzResidParams p) {
  // part blockIdx.z of gridDim.z takes chunks [z nchunk / P, (z + 1) nchunk / P) (P <= nchunk: none empty)
  const int nchunk = static_cast<int>((p.n + kKBlock * kOzChunkKB - 1) / (kKBlock * kOzChunkKB));
  const int P = static_cast<int>(gridDim.z), z = static_cast<int>(blockIdx.z);
  oz_resid_tile<RC>(&tmA, &tmX, p, static_cast<int64_t>(blockIdx.x) * kOzTile, static_cast<int>(blockIdx.y) * RC,
                    z * nchunk / P, (z + 1) * nchunk / P, P, z);
}

// The epilogue of a K-split residual: entry (i, c) adds its parts' float-float sums in part order, then
// applies the tile epilogue (R = B - a_ii x - A_offdiag x, c1 = d1 = R / a_ii, the column maximum of |R|).
// Block (x, k): rows 256 x .. + 255 of the k-th active column.
__global__ void __launch_bounds__(256) oz_finish_kernel(OzResidParams p, int nparts) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x;
  const int col = p.cols ? p.cols[blockIdx.y] : static_cast<int>(blockIdx.y);
  unsigned long long bits = 0;
  if (i < p.n) {
    float hi = 0.0f, lo = 0.0f;
    for (int z = 0; z < nparts; ++z) {
      const float2 v = p.part[(static_cast<int64_t>(z) * p.r + col) * p.ld + i];
      ff_add(hi, lo, v.x);
      ff_add(hi, lo, v.y);
    }
    const float s = __fadd_rn(hi, lo);  // renormalise: |lo| <= ulp(hi) / 2
    lo = __fsub_rn(lo, __fsub_rn(s, hi));
    hi = s;
    const int e = p.aexp[i], g = p.xexp[col];
    double dot;
    if (e == kExpNonfinite || g == kExpNonfinite)
      dot = __longlong_as_double(0x7FF8000000000000ll);
    else
      dot = scale2(static_cast<double>(hi) + static_cast<double>(lo), e + g + 2 - 16);
    const int64_t o = static_cast<int64_t>(col) * p.ld + i;
    const double r = fma(-p.d[i], p.x[o], p.b[o]) - dot;
    const float cc = static_cast<float>(r * p.rinv[i]);
    p.c1[o] = cc;
    p.d1[o] = cc;
    if (p.d1h) p.d1h[o] = __float2bfloat16_rn(cc);
    bits = abs_bits(r);
  }
  bits = warp_max_u64(bits);
  if ((threadIdx.x & 31) == 0 && bits) atomicMax(p.colmax + col, bits);
}

// Many independent residuals in one launch (the serving rounds): CTA b takes row tile b - first[k] of
// request k (first[k] <= b < first[k + 1]), all of its (at most 16) columns, with the request's two tensor
// maps at maps[2k] (A's digits) and maps[2k + 1] (X's digits).
__global__ void __launch_bounds__(OzCfg<16>::kThreads, 1)
    oz_resid_grouped_kernel(const OzResidParams* __restrict__ ps, const CUtensorMap* __restrict__ maps,
                            const int64_t* __restrict__ first, int nreq) {
  const int64_t b = blockIdx.x;
  int lo = 0, hi = nreq - 1;  // last k with first[k] <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (first[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  const OzResidParams p = ps[lo];
  if (threadIdx.x == 0) {
    // the maps were written through the generic proxy (a host copy): order that before the TMA unit reads them
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(maps + 2 * lo) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(maps + 2 * lo + 1) : "memory");
  }
  const int nchunk = static_cast<int>((p.n + kKBlock * kOzChunkKB - 1) / (kKBlock * kOzChunkKB));
  oz_resid_tile<16>(maps + 2 * lo, maps + 2 * lo + 1, p, (b - first[lo]) * kOzTile, 0, 0, nchunk, 1, 0);
}

// The X digits of many residuals: block (c, k) splits column c of request k, whose X has p.nact columns
// (zero digits for c >= nact, the padding up to kOzServeCols).
__global__ void oz_split_x_grouped_kernel(const OzResidParams* __restrict__ ps) {
  __shared__ uint32_t sh[32];
  const OzResidParams& p = ps[blockIdx.y];
  const int64_t c = blockIdx.x, n = p.n, ld = p.ld, r = p.nact;
  const double* col = p.x + c * ld;
  uint32_t m = 0;
  if (c < r)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = max(m, abs_hi(col[i]));
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  uint32_t t = 0;
  for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t = max(t, sh[w]);
  const int g = oz_exponent(t);
  if (threadIdx.x == 0) p.xexp_w[c] = g;
  for (int64_t i = threadIdx.x; i < ld; i += blockDim.x) {
    int d[kOzDigits];
    oz_digits(c < r && i < n ? col[i] : 0.0, g, d);
#pragma unroll
    for (int q = 0; q < kOzDigits; ++q) p.xd[(q * kOzServeCols + c) * ld + i] = oz_digit_value(d[q], q);
  }
}

// Parts of the K range per tile: one CTA per SM is resident (the ring takes the shared memory), so
// `tiles` CTAs fill tiles / (sms ceil(tiles / sms)) of the waves they take; splitting K into P parts makes
// tiles P CTAs of 1 / P the work.  The fewest parts whose waves are at least 2 % fuller than with fewer
// parts, at most kOzMaxParts and at most one part per chunk of K.
int oz_parts(int64_t tiles, int64_t nchunk, int sms) {
  auto fill = [&](int P) {
    const int64_t ctas = tiles * P;
    const int64_t waves = (ctas + sms - 1) / sms;
    return static_cast<double>(ctas) / static_cast<double>(waves * sms);
  };
  int best = 1;
  double bf = fill(1);
  for (int P = 2; P <= kOzMaxParts && P <= nchunk; ++P) {
    const double f = fill(P);
    if (f > bf + 0.02) {
      best = P;
      bf = f;
    }
  }
  return best;
}

template <int RC>
cudaError_t launch_resid_rc(const CUtensorMap& ta, const CUtensorMap& tx, const OzResidParams& p, cudaStream_t s) {
  constexpr int smem = OzCfg<RC>::kSmem;
  cudaError_t e = cudaFuncSetAttribute(oz_resid_kernel<RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t tiles = (p.nr / kOzTile) * (p.r / RC);
  const int64_t nchunk = (p.n + kKBlock * kOzChunkKB - 1) / (kKBlock * kOzChunkKB);
  const int P = p.part ? oz_parts(tiles, nchunk, sms) : 1;
  const dim3 grid(static_cast<unsigned>(p.nr / kOzTile), static_cast<unsigned>(p.r / RC), static_cast<unsigned>(P));
  oz_resid_kernel<RC><<<grid, OzCfg<RC>::kThreads, smem, s>>>(ta, tx, p);
  if ((e = cudaGetLastError()) != cudaSuccess || P == 1) return e;
  const int64_t ncols = p.cols ? p.nact : p.r;
  if (ncols < 1) return cudaSuccess;
  oz_finish_kernel<<<dim3(static_cast<unsigned>((p.n + 255) / 256), static_cast<unsigned>(ncols)), 256, 0, s>>>(p, P);
  return cudaGetLastError();
}

}  // namespace

bool oz_make_maps(const __nv_bfloat16* adig, const __nv_bfloat16* xdig, int64_t n, int64_t ld, CUtensorMap* maps) {
  const int64_t nr = oz_padded_rows(n);
  return make_map(&maps[0], adig, n, kOzDigits * nr, ld, kOzTile) &&
         make_map(&maps[1], xdig, n, kOzDigits * kOzServeCols, ld, kOzServeCols);
}

cudaError_t launch_oz_grouped(const OzResidParams* ps_dev, const CUtensorMap* maps_dev, const int64_t* first_dev,
                              int nreq, int64_t tiles, cudaStream_t s) {
  if (nreq < 1 || tiles < 1) return cudaSuccess;
  oz_split_x_grouped_kernel<<<dim3(kOzServeCols, static_cast<unsigned>(nreq)), 256, 0, s>>>(ps_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  constexpr int smem = OzCfg<16>::kSmem;
  e = cudaFuncSetAttribute(oz_resid_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  oz_resid_grouped_kernel<<<static_cast<unsigned>(tiles), OzCfg<16>::kThreads, smem, s>>>(ps_dev, maps_dev,
                                                                                          first_dev, nreq);
  return cudaGetLastError();
}

int64_t oz_padded_rows(int64_t n) { return (n + kOzTile - 1) / kOzTile * kOzTile; }

cudaError_t launch_oz_split_a(const double* A, int64_t lda, int64_t n, int64_t ld, __nv_bfloat16* dig, int* aexp,
                              cudaStream_t s) {
  const int64_t nr = oz_padded_rows(n);
  const int64_t blocks = std::min<int64_t>((nr + 7) / 8, 152 * 16);
  oz_split_a_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(A, lda, n, nr, ld, dig, aexp);
  return cudaGetLastError();
}

cudaError_t launch_oz_split_x(int64_t n, int64_t r, int64_t ld, const double* x, __nv_bfloat16* xd, int* xexp,
                              cudaStream_t s) {
  oz_split_x_kernel<<<static_cast<unsigned>(r), 512, 0, s>>>(n, r, ld, x, xd, xexp);
  return cudaGetLastError();
}

cudaError_t launch_oz_resid(const __nv_bfloat16* adig, const __nv_bfloat16* xdig, const OzResidParams& p,
                            cudaStream_t s) {
  if (p.r != 16 && p.r != 32 && p.r % 64 != 0) return cudaErrorInvalidValue;
  if (p.nr % kOzTile != 0 || p.ld % 16 != 0) return cudaErrorInvalidValue;
  const int rc = p.r < 64 ? static_cast<int>(p.r) : 64;
  CUtensorMap ta, tx;
  if (!make_map(&ta, adig, p.n, kOzDigits * p.nr, p.ld, kOzTile)) return cudaErrorInvalidValue;
  if (!make_map(&tx, xdig, p.n, kOzDigits * p.r, p.ld, rc)) return cudaErrorInvalidValue;
  switch (rc) {
    case 16: return launch_resid_rc<16>(ta, tx, p, s);
    case 32: return launch_resid_rc<32>(ta, tx, p, s);
    default: return launch_resid_rc<64>(ta, tx, p, s);
  }
}

}  // namespace jac
