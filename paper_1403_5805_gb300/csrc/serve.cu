// Serving: continuous batching of many independent solve requests (Section 2's Jacobi iteration with
// FP64 refinement around FP32 inner sweeps), each request up to JACOBI_SERVE_MAX_N unknowns and
// JACOBI_SERVE_MAX_RHS right-hand sides.
//
// The server keeps every admitted request's state on the device (A, its FP32 copy, X, the inner
// iterates) inside one arena whose size is the memory budget.  Work proceeds in rounds: one launch of
// serve_round_kernel advances EVERY active request by one phase (setup, FP64 residual, or one FP32 inner
// sweep), its 16-row blocks spread over all SMs as independent work items.  Between rounds the host
// reads each request's reductions, moves its state machine, retires finished requests (copying X out
// and freeing their arena space) and admits waiting ones as memory frees up, so requests that arrive
// while others run join the next round and overlap with them on the device.  A request's arithmetic
// does not depend on what else is in the round, so its result is the same alone and in the mix.
//
// Requests can bring their own A and B (device or host memory) or be generated on the device from a
// seed by serve_generate_kernel, a twin of the host generator in synth/ (Philox4x32-10, Salmon et al.
// SC'11): A with off-diagonals int32(w) 2^-31 and a_ii = f * sum_{j != i} |a_ij| * (+-1), B uniform.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <type_traits>
#include <vector>

#include "device_util.cuh"
#include "f64tof32.cuh"
#include "mrhs.cuh"
#include "solver.cuh"
#include "splitfloat.cuh"

namespace jac {
namespace {

constexpr int kSRows = 16;        // rows per work item
constexpr int kSRhs = 16;         // right-hand sides per request (JACOBI_SERVE_MAX_RHS)
constexpr int kKC = 256;          // columns of the iterate staged in shared memory per step
constexpr int kSThreads = 256;    // 8 warps x 2 rows
constexpr int kPrepSteps = 4;     // setup: 128-column steps of a row whose loads are in flight together
constexpr int kStatSlots = 64;    // per request per round: [0,16) |R| or change per column, [16,32) |B|,
                                  // 32 inner change, 33 inner magnitude, 34 bad-diagonal key (~key),
                                  // [40,56) max |b / a_ii| per column (setup round)

enum SrvPhase : int { kPhPrep = 0, kPhResid = 1, kPhInner = 2 };

struct SrvReq {
  int64_t n, r, ld;
  const double* A;   // n x n row-major, row stride ld (rows 128-byte aligned; padding never read)
  float* Nl;         // FP32 copy of the off-diagonal part, row stride ld
  double* d;
  double* rinv;
  float* rowfac;
  const double* B;   // [r][ld]
  double* X[2];      // FP64 iterate buffers [r][ld]
  float* C1;         // inner right-hand side [r][ld]
  float* D[2];       // inner iterates [r][ld]
  unsigned long long* st;  // kStatSlots reduction slots (zeroed every round)
  // split-float residual (split != 0): per-row scale exponents of A, the two FP32 words of X[k] 2^-g_c
  // per entry, and the column exponents g_c (from max_i |b_ic / a_ii|)
  int* rexp;
  float2* xs[2];
  int xg[16];
  int phase, xsel, dsel, rb, split;
  // tensor-core residual (JACOBI_FLAG_TC_RESIDUAL): A's digit matrices and row exponents (written at
  // admission), X's digits and column exponents (written by each residual round)
  __nv_bfloat16* adig;
  int* aexp;
  __nv_bfloat16* xdig;
  int* xexp;
};

// ------------------------------------------------------------------------ Philox4x32-10 (device)
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Block q of the sequence (seed, stream): the four words 4q .. 4q + 3, counter (q, stream, 0).
__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint32_t stream, uint64_t q) {
  return philox(make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32), stream, 0u),
                make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
}

// Word w of the sequence (seed, stream): lane w % 4 of the block with counter (w / 4, stream, 0).
__device__ __forceinline__ uint32_t philox_word(uint64_t seed, uint32_t stream, uint64_t w) {
  const uint4 o = philox_block(seed, stream, w >> 2);
  switch (w & 3) {
    case 0: return o.x;
    case 1: return o.y;
    case 2: return o.z;
    default: return o.w;
  }
}

// int32(word) * 2^-31 (exact), assembled from the bits on the integer units: on GB300 an int -> double
// conversion and a double multiply each take the FP64 pipe, which the residual rounds need.
__device__ __forceinline__ double signed_unit(uint32_t word) {
  const int32_t w = static_cast<int32_t>(word);
  if (w == 0) return 0.0;
  const uint32_t u = w < 0 ? 0u - word : word;  // |w|, 1 .. 2^31
  const int lz = __clz(u);                      // |w| in [2^(31 - lz), 2^(32 - lz))
  const uint64_t frac = (static_cast<uint64_t>(u) << (21 + lz)) & 0xFFFFFFFFFFFFFull;
  const uint64_t bits = (static_cast<uint64_t>(w < 0) << 63) | (static_cast<uint64_t>(1023 - lz) << 52) | frac;
  return __longlong_as_double(static_cast<long long>(bits));
}

// One CTA per row (grid-stride): A row i (row stride lda), its diagonal, and B (column stride ld).
__global__ void serve_generate_kernel(int64_t n, int64_t r, int64_t lda, int64_t ld, double f, uint64_t seed,
                                      double* A, double* B) {
  __shared__ unsigned long long part[kSThreads / 32];
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    // sum_{j != i} |a_ij| 2^31 as an integer (below 2^44): exactly the FP64 sum of the |a_ij|, in any order
    unsigned long long s = 0;
    // words i n .. i n + n - 1 of stream 0, one Philox block (4 words) per thread and step
    const uint64_t w0 = static_cast<uint64_t>(i * n), w1 = w0 + static_cast<uint64_t>(n);
    for (uint64_t q = (w0 >> 2) + threadIdx.x; 4 * q < w1; q += blockDim.x) {
      const uint4 o = philox_block(seed, 0u, q);
      const uint32_t words[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const uint64_t w = 4 * q + e;
        if (w < w0 || w >= w1) continue;
        const int64_t j = static_cast<int64_t>(w - w0);
        if (j == i) continue;
        A[i * lda + j] = signed_unit(words[e]);
        const int32_t v = static_cast<int32_t>(words[e]);
        s += v < 0 ? 0u - words[e] : words[e];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tot = 0;
      for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) tot += part[w];
      const double t = static_cast<double>(tot) * 0x1p-31;
      const double sign = (philox_word(seed, 1u, static_cast<uint64_t>(i)) & 1u) ? -1.0 : 1.0;
      A[i * lda + i] = n > 1 ? f * t * sign : f * sign;
    }
    __syncthreads();
    for (int64_t c = threadIdx.x; c < r; c += blockDim.x)
      B[c * ld + i] = signed_unit(philox_word(seed, 5u, static_cast<uint64_t>(c * n + i)));
  }
}

// ------------------------------------------------------------------------------- round kernel
template <int R, int OFF, typename Acc>
struct TRs {
  static __device__ __forceinline__ Acc run(const Acc (&v)[R], int lane) {
    constexpr int H = R / 2;
    Acc w[H];
    const bool hi = lane & OFF;
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const Acc send = hi ? v[q] : v[q + H];
      const Acc keep = hi ? v[q + H] : v[q];
      w[q] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
    }
    return TRs<H, OFF / 2, Acc>::run(w, lane);
  }
};
template <int OFF, typename Acc>
struct TRs<1, OFF, Acc> {
  static __device__ __forceinline__ Acc run(const Acc (&v)[1], int) { return v[0]; }
};
// After TRs<V, 16>, lanes sharing bits [4 .. 5 - log2 V] hold value index (those bits); finish the sum
// over the remaining low lane bits.
template <int V, typename Acc>
__device__ __forceinline__ Acc tr_finish(Acc w) {
#pragma unroll
  for (int o = 16 / V; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  return w;
}
template <int V>
__device__ __forceinline__ int tr_index(int lane) {
  int idx = 0, bit = 4;
#pragma unroll
  for (int k = V; k > 1; k >>= 1, --bit) idx = (idx << 1) | ((lane >> bit) & 1);
  return idx;
}

__device__ __forceinline__ void umax_to(unsigned long long* p, unsigned long long v) {
  if (v) atomicMax(p, v);
}

// Setup of rows [i0, i0 + 2) handled by one warp: diagonal and reciprocals, FP32 copy of the off-
// diagonal row (4 consecutive elements per lane and step: A's rows start 128-byte aligned), the first
// inner right-hand side C1 = B / a_ii (the residual of X = 0) and D0 = C1.
__device__ void prep_rows(const SrvReq& q, int64_t i0, int lane) {
  const int64_t n = q.n, ld = q.ld;
  for (int rr = 0; rr < 2; ++rr) {
    const int64_t i = i0 + rr;
    if (i >= n) break;
    const double* Ai = q.A + i * ld;
    float* Ni = q.Nl + i * ld;
    uint32_t mb = 0;  // max_j of the high word of |a_ij|
    // kPrepSteps steps of 128 columns per pass: all of their loads are issued before the conversions, so
    // a warp keeps that many 32-byte loads per lane in flight
    for (int64_t jb = 4 * lane; jb < ld; jb += 128 * kPrepSteps) {
      double a[kPrepSteps][4];
#pragma unroll
      for (int u = 0; u < kPrepSteps; ++u) {
        const int64_t j = jb + 128 * u;
        if (j + 4 <= n) {
          const double2 v0 = __ldcs(reinterpret_cast<const double2*>(Ai + j));
          const double2 v1 = __ldcs(reinterpret_cast<const double2*>(Ai + j + 2));
          a[u][0] = v0.x;
          a[u][1] = v0.y;
          a[u][2] = v1.x;
          a[u][3] = v1.y;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) a[u][e] = j + e < n ? Ai[j + e] : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < kPrepSteps; ++u) {
        const int64_t j = jb + 128 * u;
        if (j < ld) {
          float f[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            mb = max(mb, abs_hi(a[u][e]));
            f[e] = (j + e < n && j + e != i) ? f64_to_f32_rn(a[u][e]) : 0.0f;  // off the FP64 pipe
          }
          *reinterpret_cast<float4*>(Ni + j) = make_float4(f[0], f[1], f[2], f[3]);
        }
      }
    }
    if (q.split) {
      mb = __reduce_max_sync(0xffffffffu, mb);
      if (lane == 0) q.rexp[i] = split_exponent_hi(mb);
    }
    const double a = Ai[i];
    const double ri = (a != 0.0 && isfinite(a)) ? __drcp_rn(a) : 0.0;
    if (lane == 0) {
      q.d[i] = a;
      q.rinv[i] = ri;
      q.rowfac[i] = __double2float_rn(ri);
      if (!isfinite(a) || a == 0.0)
        atomicMax(q.st + 34, ~((static_cast<unsigned long long>(i) << 8) | (isfinite(a) ? 2ull : 3ull)));
    }
    for (int64_t c = lane; c < q.r; c += 32) {
      const double b = q.B[c * ld + i];
      const float cc = static_cast<float>(b * ri);
      q.C1[c * ld + i] = cc;
      q.D[0][c * ld + i] = cc;
      umax_to(q.st + 16 + c, abs_bits(b));
      umax_to(q.st + 40 + c, abs_bits(b * ri));
    }
  }
}

// Elements j, j + 1 (j even) of a row whose start is 16-byte aligned; entries at or past n are 0 and
// not loaded.
__device__ __forceinline__ double2 load_pair(const double* row, int64_t j, int64_t n) {
  if (j + 1 < n) return __ldcs(reinterpret_cast<const double2*>(row + j));
  return make_double2(j < n ? row[j] : 0.0, 0.0);
}

// Shared memory of one round CTA: the staged chunk of the iterate (FP64 X, its split words, or the
// FP32 inner iterate D; kSRhs columns x kKC entries) and the cross-warp partial sums of the inner sweep.
constexpr int kIStages = 3;  // chunks of the inner sweep in flight (asynchronous copies)
struct SrvSmem {
  union {
    double x[kSRhs][kKC];
    float2 xs[kSRhs][kKC];
    struct {
      // the item's rows of the narrow matrix, one chunk per stage; one quad of padding per row puts the
      // 16 rows of a quad column on different banks
      float4 a[kIStages][kSRows][kKC / 4 + 1];
      float4 d[kIStages][kSRhs][kKC / 4];  // D_cur, one chunk per stage
    } in;
    float part[kSThreads / 32][kSRows][kSRhs];  // inner sweep: each warp's row sums, after the chunks
  };
};

// 16-byte asynchronous copy global -> shared (cp.async, the L2-only form); with valid == false nothing is
// read and the 16 bytes are zero-filled.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Waits until at most N of this thread's most recent copy groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage entries [j0, j0 + kKC) of r columns of a [r][ld] vector block (zero past ld) into shared memory.
template <typename T>
__device__ __forceinline__ void stage_cols(const T* __restrict__ v, int64_t r, int64_t ld, int64_t j0,
                                           T (*dst)[kKC]) {
  for (int e = threadIdx.x; e < static_cast<int>(r) * kKC; e += kSThreads) {
    const int c = e / kKC, jj = e % kKC;
    dst[c][jj] = j0 + jj < ld ? v[c * ld + j0 + jj] : T{};
  }
}

// Residual R = B - A X of the work item's rows r0 + 2 warp + {0, 1} for RB >= r columns: FP64 FMAs, or
// (kSplit) the split-float arithmetic of splitfloat.cuh on the FP32 units.  X is staged per CTA in
// chunks of kKC columns; every warp takes part in the staging, also when its rows are past n.  The FP64
// form accumulates both rows in one pass; the split form takes one row per pass (its float-float
// accumulators are twice as wide), staging X once per pass.
template <int RB, bool kSplit>
__device__ void resid_item(const SrvReq& q, int64_t r0, int warp, int lane, SrvSmem& sm) {
  using Acc = typename std::conditional<kSplit, FF, double>::type;
  constexpr int RP = kSplit ? 1 : 2;  // rows per pass
  const int64_t n = q.n, ld = q.ld, i0 = r0 + 2 * warp;
  const int r = static_cast<int>(q.r);
  for (int pass = 0; pass < 2 / RP; ++pass) {
    const int64_t ia = i0 + RP * pass;  // first row of this pass
    const bool has0 = ia < n, has1 = RP == 2 && ia + 1 < n;
    const double* A0 = q.A + (has0 ? ia : 0) * ld;
    const double* A1 = q.A + (has1 ? ia + 1 : 0) * ld;
    const int sh0 = kSplit && has0 ? q.rexp[ia] : 0;
    Acc acc[RP * RB];
#pragma unroll
    for (int v = 0; v < RP * RB; ++v) acc[v] = Acc{};
    for (int64_t j0 = 0; j0 < n; j0 += kKC) {
      __syncthreads();  // the previous chunk is consumed
      if constexpr (kSplit)
        stage_cols(q.xsel ? q.xs[1] : q.xs[0], r, ld, j0, sm.xs);
      else
        stage_cols(q.xsel ? q.X[1] : q.X[0], r, ld, j0, sm.x);
      __syncthreads();
      if (has0) {
        // lane l takes columns 2 l + 64 t (t < kKC / 64) of the chunk: all of its A loads (16 bytes each,
        // rows are 128-byte aligned) are issued before the arithmetic; columns past n read as 0 (the
        // row padding is never read)
        double2 a0v[kKC / 64], a1v[kKC / 64];
#pragma unroll
        for (int t = 0; t < kKC / 64; ++t) {
          const int64_t j = j0 + 2 * lane + 64 * t;
          a0v[t] = load_pair(A0, j, n);
          a1v[t] = has1 ? load_pair(A1, j, n) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int t = 0; t < kKC / 64; ++t) {
          const int jp = lane + 32 * t;  // index of the column pair in the chunk
          if constexpr (kSplit) {
            float h0, l0, h1, l1;
            split_scaled(a0v[t].x, sh0, h0, l0);
            split_scaled(a0v[t].y, sh0, h1, l1);
#pragma unroll
            for (int c = 0; c < RB; ++c)
              if (c < r) {
                const float4 x = reinterpret_cast<const float4*>(sm.xs[c])[jp];
                ff_fma(acc[c], h0, l0, x.x, x.y);
                ff_fma(acc[c], h1, l1, x.z, x.w);
              }
          } else {
#pragma unroll
            for (int c = 0; c < RB; ++c)
              if (c < r) {
                const double2 x = reinterpret_cast<const double2*>(sm.x[c])[jp];
                acc[c] = fma(a0v[t].y, x.y, fma(a0v[t].x, x.x, acc[c]));
                acc[RB + c] = fma(a1v[t].y, x.y, fma(a1v[t].x, x.x, acc[RB + c]));
              }
          }
        }
        if constexpr (kSplit) {
#pragma unroll
          for (int v = 0; v < RB; ++v) ff_renorm(acc[v]);
        }
      }
    }
    if (!has0) continue;  // warp-uniform; the next pass (if any) has no valid row either
    // one transposed reduction per row (RB values each), FP64 across lanes
#pragma unroll
    for (int rr = 0; rr < RP; ++rr) {
      double dv[RB];
#pragma unroll
      for (int c = 0; c < RB; ++c) {
        if constexpr (kSplit)
          dv[c] = static_cast<double>(acc[rr * RB + c].hi) + static_cast<double>(acc[rr * RB + c].lo);
        else
          dv[c] = acc[rr * RB + c];
      }
      const double tot = tr_finish<RB>(TRs<RB, 16, double>::run(dv, lane));
      const int c = tr_index<RB>(lane);
      const int64_t i = ia + rr;
      if ((lane & (32 / RB - 1)) == 0 && i < n && c < r) {
        const int64_t o = c * ld + i;
        const double dot = kSplit ? tot * pow2(sh0) * pow2(q.xg[c]) : tot;
        const double R = q.B[o] - dot;
        const float cc = static_cast<float>(R * q.rinv[i]);
        q.C1[o] = cc;
        q.D[0][o] = cc;
        umax_to(q.st + c, abs_bits(R));
      }
    }
  }
}

// Issues the asynchronous copies of chunk j0 of the inner sweep into stage st: the item's 16 rows of the
// narrow matrix (rows past n zero-filled; the narrow rows are zero-padded up to ld, so whole quads below ld
// are read) and the r staged columns of D_cur; then closes the copy group.  Each thread copies 4 quads of
// the rows and up to 4 of D.
__device__ __forceinline__ void inner_issue(const SrvReq& q, const float* Dc, int64_t r0, int64_t j0, int st,
                                            SrvSmem& sm) {
  const int64_t n = q.n, ld = q.ld;
  const int nq = static_cast<int>(q.r) * (kKC / 4);
#pragma unroll
  for (int k = 0; k < kSRows * (kKC / 4) / kSThreads; ++k) {
    const int e = threadIdx.x + k * kSThreads;
    const int row = e / (kKC / 4), q4 = e % (kKC / 4);
    const int64_t i = r0 + row, j = j0 + 4 * q4;
    const bool ok = i < n && j < ld;
    cp_async16(&sm.in.a[st][row][q4], ok ? q.Nl + i * ld + j : q.Nl, ok);
  }
#pragma unroll
  for (int k = 0; k < kSRhs * (kKC / 4) / kSThreads; ++k) {
    const int e = threadIdx.x + k * kSThreads;
    if (e < nq) {
      const int c = e / (kKC / 4), q4 = e % (kKC / 4);
      const int64_t j = j0 + 4 * q4;
      cp_async16(&sm.in.d[st][c][q4], j < ld ? Dc + c * ld + j : Dc, j < ld);
    }
  }
  cp_async_commit();
}

// FP32 inner sweep of the work item's 16 rows: D_new = C1 - (1/a_ii) N D_cur, X_alt = X_cur + D_new.
// The item's rows of N and the iterate D_cur stream through shared memory in chunks of kKC columns by
// asynchronous copies, kIStages chunks in flight, so the loads of the next chunks overlap the arithmetic
// of this one (one barrier per chunk).  Lane 16 h + t of warp w takes row t of the item and, in step s of
// a chunk, quad 16 s + 2 w + h: the 16 lanes of a half-warp read the same D_cur quads (a broadcast), so
// each quad of D read from shared memory feeds 16 rows.  Each lane accumulates its row for every
// right-hand side; the two halves and then the 8 warps are added in a fixed order.
template <int RB>
__device__ void inner_item(const SrvReq& q, int64_t r0, int warp, int lane, SrvSmem& sm) {
  constexpr int kWarps = kSThreads / 32;
  constexpr int kSteps = (kKC / 4) / (2 * kWarps);  // quads of a chunk per lane
  static_assert(kSteps * 2 * kWarps == kKC / 4, "the warps' quads tile a chunk");
  static_assert(kIStages == 3, "the copy-group accounting below keeps two chunks ahead");
  static_assert(RB * kSRows <= kSThreads, "one thread per (row, right-hand side) in the epilogue");
  const int t = lane & 15, h = lane >> 4;
  const int64_t n = q.n, ld = q.ld;
  float acc[RB];
#pragma unroll
  for (int c = 0; c < RB; ++c) acc[c] = 0.0f;
  const float* Dc = q.dsel ? q.D[1] : q.D[0];
  const int64_t nch = (n + kKC - 1) / kKC;
  // the previous item's readers of shared memory passed the barrier that ends it
  inner_issue(q, Dc, r0, 0, 0, sm);
  if (nch > 1)
    inner_issue(q, Dc, r0, kKC, 1, sm);
  else
    cp_async_commit();  // an empty group keeps the count of groups in flight the same
#pragma unroll 1
  for (int64_t ch = 0; ch < nch; ++ch) {
    const int st = static_cast<int>(ch % kIStages);
    cp_async_wait<1>();  // this thread's copies of chunk ch have landed
    __syncthreads();     // everyone's have; every reader of the stage chunk ch + 2 reuses is done
    if (ch + 2 < nch)
      inner_issue(q, Dc, r0, (ch + 2) * kKC, static_cast<int>((ch + 2) % kIStages), sm);
    else
      cp_async_commit();
    const int64_t j0 = ch * kKC;
#pragma unroll
    for (int s = 0; s < kSteps; ++s) {
      const int q4 = 2 * kWarps * s + 2 * warp + h;
      if (j0 + 4 * q4 < n) {
        const float4 m = sm.in.a[st][t][q4];
#pragma unroll
        for (int c = 0; c < RB; ++c)
          if (c < q.r) {
            const float4 x = sm.in.d[st][c][q4];
            acc[c] = fmaf(m.x, x.x, fmaf(m.y, x.y, fmaf(m.z, x.z, fmaf(m.w, x.w, acc[c]))));
          }
      }
    }
  }
  cp_async_wait<0>();  // only empty groups remain; nothing is left in flight
#pragma unroll
  for (int c = 0; c < RB; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 16);
  __syncthreads();  // the stages are read; part aliases them
  if (h == 0) {
#pragma unroll
    for (int c = 0; c < RB; ++c) sm.part[warp][t][c] = acc[c];
  }
  __syncthreads();
  unsigned long long chg = 0, mag = 0;
  const int row = threadIdx.x / RB, c = threadIdx.x % RB;
  const int64_t i = r0 + row;
  if (row < kSRows && i < n && c < q.r) {
    float sum = sm.part[0][row][c];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) sum += sm.part[w][row][c];  // fixed order
    const int64_t o = c * ld + i;
    const float val = fmaf(-q.rowfac[i], sum, q.C1[o]);
    const float old = Dc[o];
    (q.dsel ? q.D[0] : q.D[1])[o] = val;
    const double xn = (q.xsel ? q.X[1] : q.X[0])[o] + static_cast<double>(val);
    (q.xsel ? q.X[0] : q.X[1])[o] = xn;
    if (q.split) (q.xsel ? q.xs[0] : q.xs[1])[o] = split_x(xn, q.xg[c]);
    chg = abs_bits(val - old);
    mag = abs_bits(val);
  }
  chg = warp_max_u64(chg);
  mag = warp_max_u64(mag);
  if (lane == 0) {
    umax_to(q.st + 32, chg);
    umax_to(q.st + 33, mag);
  }
}

template <int RB>
__device__ __forceinline__ void run_item(const SrvReq& q, int64_t r0, int warp, int lane, SrvSmem& sm) {
  if (q.phase == kPhResid) {
    if (q.split)
      resid_item<RB, true>(q, r0, warp, lane, sm);
    else
      resid_item<RB, false>(q, r0, warp, lane, sm);
  } else {
    inner_item<RB>(q, r0, warp, lane, sm);
  }
}

// Work items are handed out by an atomic counter (*queue, zero at launch) in array order; the host orders
// the requests by the cost of one of their items, heaviest first, so the long items start early and the
// short ones fill the end of the round.
__global__ void __launch_bounds__(kSThreads, 2) serve_round_kernel(const SrvReq* __restrict__ reqs, int nreq,
                                                                   const int64_t* __restrict__ first, int64_t items,
                                                                   unsigned long long* queue) {
  extern __shared__ __align__(16) unsigned char srv_dyn_smem[];
  SrvSmem& sm = *reinterpret_cast<SrvSmem*>(srv_dyn_smem);
  __shared__ long long s_item;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) s_item = static_cast<long long>(atomicAdd(queue, 1ull));
    __syncthreads();
    const int64_t it = s_item;
    if (it >= items) break;
    int lo = 0, hi = nreq - 1;  // request owning this item: last k with first[k] <= it
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (first[mid] <= it)
        lo = mid;
      else
        hi = mid - 1;
    }
    const SrvReq& q = reqs[lo];  // fields read on demand (L1); dynamic indexing stays off the stack
    const int64_t r0 = (it - first[lo]) * kSRows;  // CTA-uniform
    if (q.phase == kPhPrep) {
      const int64_t i0 = r0 + 2 * warp;
      if (i0 < q.n) prep_rows(q, i0, lane);
      __syncthreads();  // s_item is rewritten by the next claim
      continue;
    }
    switch (q.rb) {
      case 1: run_item<1>(q, r0, warp, lane, sm); break;
      case 2: run_item<2>(q, r0, warp, lane, sm); break;
      case 4: run_item<4>(q, r0, warp, lane, sm); break;
      case 8: run_item<8>(q, r0, warp, lane, sm); break;
      default: run_item<16>(q, r0, warp, lane, sm); break;
    }
    __syncthreads();  // the next item restages shared memory (and s_item)
  }
}

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace jac

using namespace jac;

namespace {

// First-fit allocator over the arena (host-side bookkeeping of device offsets).
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free;  // offset -> bytes
  void reset(size_t bytes) {
    size = bytes;
    free.clear();
    free[0] = bytes;
  }
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = free.begin(); it != free.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free.erase(it);
        if (rest) free[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto it = free.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free.erase(nx);
    }
    if (it != free.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free.erase(it);
      }
    }
  }
};

struct Request {
  int64_t id = 0, n = 0, r = 0, ld = 0;
  double f = 0.0;
  uint64_t seed = 0;
  bool generate = false;
  const double* A_in = nullptr;
  const double* B_in = nullptr;
  double* X_out = nullptr;
  size_t off = 0, bytes = 0;
  SrvReq q{};
  int64_t outer = 0, inner_total = 0, inner_step = 0;
  std::vector<double> bnorm;  // ||b_c||_inf per column (from the setup round)
  jacobi_stats st{};
  CUtensorMap maps[2];        // tensor-core residual: TMA maps of A's and X's digits
  bool maps_ok = true;
};

size_t request_bytes(int64_t n, int64_t r, int64_t ld, bool own_A, bool split, bool tc) {
  size_t b = 0;
  if (tc) {
    const int64_t nr = oz_padded_rows(n);
    b += a256(static_cast<size_t>(kOzDigits) * nr * ld * 2) + a256(static_cast<size_t>(nr) * 4);
    b += a256(static_cast<size_t>(kOzDigits) * kOzServeCols * ld * 2) + a256(kOzServeCols * 4);
  }
  if (own_A) b += a256(static_cast<size_t>(n) * ld * 8);    // A, rows padded to ld (128-byte aligned)
  b += a256(static_cast<size_t>(n) * ld * 4);                // Nl
  b += 2 * a256(static_cast<size_t>(ld) * 8) + a256(static_cast<size_t>(ld) * 4);  // d, rinv, rowfac
  b += 3 * a256(static_cast<size_t>(r) * ld * 8);             // B, X0, X1
  b += 3 * a256(static_cast<size_t>(r) * ld * 4);             // C1, D0, D1
  if (split) b += a256(static_cast<size_t>(ld) * 4) + 2 * a256(static_cast<size_t>(r) * ld * 8);  // rexp, xs
  return b;
}

// Host twin of split_exponent: e with |v| < 2^e for the IEEE bits of max |v|, clamped to [-1000, 1000].
int host_split_exponent(unsigned long long bits) {
  const int be = static_cast<int>((bits >> 52) & 0x7FFu);
  if (be == 0x7FF || bits == 0) return 0;
  const int e = be == 0 ? -1000 : be - 1022;
  return e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
}

}  // namespace

struct jacobi_server {
  cudaStream_t stream = nullptr;
  char* arena_base = nullptr;
  Arena arena;
  double tol = 1e-10;
  int64_t max_iter = 5000;
  int max_inner = 1000, max_outer = 30;
  float inner_rtol = 1.0f / 1024;
  int max_active = 0;
  bool split = false;
  bool tc = false;  // residual rounds on the tensor cores (digit split)
  int64_t next_id = 1;
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::vector<std::pair<int64_t, jacobi_stats>> done;
  // per-round device / pinned buffers
  SrvReq* d_reqs = nullptr;
  int64_t* d_first = nullptr;
  unsigned long long* d_queue = nullptr;  // work-item counter of the round kernel
  // tensor-core residual rounds: per residual request its parameters, its two TMA maps and first tile
  OzResidParams* d_ozp = nullptr;
  CUtensorMap* d_maps = nullptr;
  int64_t* d_ozfirst = nullptr;
  int* d_cols = nullptr;      // 0 .. kOzServeCols - 1: the active columns of a request are its first r
  int* d_tcstat = nullptr;    // timeout code of the tensor-core residual
  OzResidParams* h_ozp = nullptr;
  CUtensorMap* h_maps = nullptr;
  int64_t* h_ozfirst = nullptr;
  int* h_tcstat = nullptr;
  unsigned long long* d_stats = nullptr;
  SrvReq* h_reqs = nullptr;
  int64_t* h_first = nullptr;
  unsigned long long* h_stats = nullptr;
  int cap = 0;
  int grid = 0;
  int64_t rounds = 0;
};

namespace {

int grow(jacobi_server* s, int need) {
  if (need <= s->cap) return JACOBI_OK;
  int cap = std::max(need, 2 * s->cap + 64);
  cudaFree(s->d_reqs);
  cudaFree(s->d_first);
  cudaFree(s->d_stats);
  cudaFreeHost(s->h_reqs);
  cudaFreeHost(s->h_first);
  cudaFreeHost(s->h_stats);
  if (cudaMalloc(&s->d_reqs, sizeof(SrvReq) * cap) != cudaSuccess ||
      cudaMalloc(&s->d_first, sizeof(int64_t) * (cap + 1)) != cudaSuccess ||
      cudaMalloc(&s->d_stats, sizeof(unsigned long long) * kStatSlots * cap) != cudaSuccess ||
      cudaMallocHost(&s->h_reqs, sizeof(SrvReq) * cap) != cudaSuccess ||
      cudaMallocHost(&s->h_first, sizeof(int64_t) * (cap + 1)) != cudaSuccess ||
      cudaMallocHost(&s->h_stats, sizeof(unsigned long long) * kStatSlots * cap) != cudaSuccess)
    return JACOBI_ERR_OUT_OF_MEMORY;
  if (s->tc) {
    cudaFree(s->d_ozp);
    cudaFree(s->d_maps);
    cudaFree(s->d_ozfirst);
    cudaFreeHost(s->h_ozp);
    cudaFreeHost(s->h_maps);
    cudaFreeHost(s->h_ozfirst);
    if (cudaMalloc(&s->d_ozp, sizeof(OzResidParams) * cap) != cudaSuccess ||
        cudaMalloc(&s->d_maps, sizeof(CUtensorMap) * 2 * cap) != cudaSuccess ||
        cudaMalloc(&s->d_ozfirst, sizeof(int64_t) * (cap + 1)) != cudaSuccess ||
        cudaMallocHost(&s->h_ozp, sizeof(OzResidParams) * cap) != cudaSuccess ||
        cudaMallocHost(&s->h_maps, sizeof(CUtensorMap) * 2 * cap) != cudaSuccess ||
        cudaMallocHost(&s->h_ozfirst, sizeof(int64_t) * (cap + 1)) != cudaSuccess)
      return JACOBI_ERR_OUT_OF_MEMORY;
  }
  s->cap = cap;
  return JACOBI_OK;
}

double as_double(unsigned long long u) {
  double v;
  std::memcpy(&v, &u, 8);
  return v;
}

int rbucket(int64_t r) { return r <= 1 ? 1 : r <= 2 ? 2 : r <= 4 ? 4 : r <= 8 ? 8 : 16; }

// Admit one request: carve its arena block, lay out its buffers, fill A and B, set phase PREP.
bool admit(jacobi_server* s, Request* rq) {
  const bool own_A = true;  // A always lives in the arena (copied or generated), row stride ld
  rq->ld = round_up(rq->n, kLdAlign);
  rq->bytes = request_bytes(rq->n, rq->r, rq->ld, own_A, s->split, s->tc);
  if (!s->arena.alloc(rq->bytes, &rq->off)) return false;
  char* p = s->arena_base + rq->off;
  SrvReq& q = rq->q;
  q = SrvReq{};
  q.n = rq->n;
  q.r = rq->r;
  q.ld = rq->ld;
  auto take = [&p](size_t bytes) {
    char* at = p;
    p += a256(bytes);
    return at;
  };
  const int64_t n = rq->n, r = rq->r, ld = rq->ld;
  double* A = reinterpret_cast<double*>(take(static_cast<size_t>(n) * ld * 8));
  q.A = A;
  q.Nl = reinterpret_cast<float*>(take(static_cast<size_t>(n) * ld * 4));
  q.d = reinterpret_cast<double*>(take(static_cast<size_t>(ld) * 8));
  q.rinv = reinterpret_cast<double*>(take(static_cast<size_t>(ld) * 8));
  q.rowfac = reinterpret_cast<float*>(take(static_cast<size_t>(ld) * 4));
  double* B = reinterpret_cast<double*>(take(static_cast<size_t>(r) * ld * 8));
  q.B = B;
  q.X[0] = reinterpret_cast<double*>(take(static_cast<size_t>(r) * ld * 8));
  q.X[1] = reinterpret_cast<double*>(take(static_cast<size_t>(r) * ld * 8));
  q.C1 = reinterpret_cast<float*>(take(static_cast<size_t>(r) * ld * 4));
  q.D[0] = reinterpret_cast<float*>(take(static_cast<size_t>(r) * ld * 4));
  q.D[1] = reinterpret_cast<float*>(take(static_cast<size_t>(r) * ld * 4));
  char* vec_end = reinterpret_cast<char*>(q.D[1]) + a256(static_cast<size_t>(r) * ld * 4);
  q.split = s->split ? 1 : 0;
  if (s->split) {
    q.xs[0] = reinterpret_cast<float2*>(take(static_cast<size_t>(r) * ld * 8));
    q.xs[1] = reinterpret_cast<float2*>(take(static_cast<size_t>(r) * ld * 8));
    vec_end = reinterpret_cast<char*>(q.xs[1]) + a256(static_cast<size_t>(r) * ld * 8);
    q.rexp = reinterpret_cast<int*>(take(static_cast<size_t>(ld) * 4));
  }
  if (s->tc) {
    const int64_t nr = oz_padded_rows(n);
    q.adig = reinterpret_cast<__nv_bfloat16*>(take(static_cast<size_t>(kOzDigits) * nr * ld * 2));
    q.aexp = reinterpret_cast<int*>(take(static_cast<size_t>(nr) * 4));
    q.xdig = reinterpret_cast<__nv_bfloat16*>(take(static_cast<size_t>(kOzDigits) * kOzServeCols * ld * 2));
    q.xexp = reinterpret_cast<int*>(take(kOzServeCols * 4));
  }
  // vectors start at zero so every padding entry is 0 (X0 = 0 is the start vector)
  const size_t vec_bytes = static_cast<size_t>(vec_end - reinterpret_cast<char*>(B));
  cudaMemsetAsync(B, 0, vec_bytes, s->stream);
  if (rq->generate) {
    int64_t blocks = std::min<int64_t>(n, 4096);
    serve_generate_kernel<<<static_cast<unsigned>(blocks), kSThreads, 0, s->stream>>>(n, r, ld, ld, rq->f, rq->seed,
                                                                                       A, B);
  } else {
    cudaMemcpy2DAsync(A, ld * 8, rq->A_in, n * 8, n * 8, n, cudaMemcpyDefault, s->stream);
    cudaMemcpy2DAsync(B, ld * 8, rq->B_in, n * 8, n * 8, r, cudaMemcpyDefault, s->stream);
  }
  if (s->tc) {
    // A's digits for the tensor-core residual rounds, and the TMA maps of both digit blocks
    launch_oz_split_a(A, ld, n, ld, q.adig, q.aexp, s->stream);
    rq->maps_ok = oz_make_maps(q.adig, q.xdig, n, ld, rq->maps);
  }
  q.phase = kPhPrep;
  q.xsel = 0;
  q.dsel = 0;
  q.rb = rbucket(r);
  rq->st = jacobi_stats{};
  rq->st.rel_residual = std::nan("");
  rq->outer = rq->inner_total = rq->inner_step = 0;
  return true;
}

void retire(jacobi_server* s, Request* rq, int status) {
  rq->st.status = status;
  rq->st.converged = status == JACOBI_OK;
  rq->st.sweeps = rq->inner_total;
  rq->st.outer_steps = rq->outer;
  if (status >= 0 && rq->X_out)
    cudaMemcpy2DAsync(rq->X_out, rq->n * 8, rq->q.X[rq->q.xsel], rq->ld * 8, rq->n * 8, rq->r, cudaMemcpyDefault,
                      s->stream);
  s->arena.release(rq->off, rq->bytes);
  s->done.emplace_back(rq->id, rq->st);
  delete rq;
}

}  // namespace

extern "C" {

int jacobi_server_create(const jacobi_server_desc* d, jacobi_server** out) {
  if (!out || !d || d->budget_bytes < (1u << 20)) return JACOBI_ERR_INVALID_ARG;
  *out = nullptr;
  jacobi_server* s = new (std::nothrow) jacobi_server();
  if (!s) return JACOBI_ERR_OUT_OF_MEMORY;
  s->stream = static_cast<cudaStream_t>(d->stream);
  if (d->tol > 0) s->tol = d->tol;
  if (d->max_iter > 0) s->max_iter = d->max_iter;
  if (d->max_inner > 0) s->max_inner = d->max_inner;
  if (d->max_outer > 0) s->max_outer = d->max_outer;
  if (d->inner_rtol > 0) s->inner_rtol = static_cast<float>(d->inner_rtol);
  s->max_active = d->max_active;
  s->split = (d->flags & JACOBI_FLAG_SPLIT_RESIDUAL) != 0;
  s->tc = (d->flags & JACOBI_FLAG_TC_RESIDUAL) != 0;
  if (s->split && s->tc) {
    delete s;
    return JACOBI_ERR_INVALID_ARG;
  }
  if (cudaMalloc(&s->arena_base, d->budget_bytes) != cudaSuccess) {
    delete s;
    return JACOBI_ERR_OUT_OF_MEMORY;
  }
  s->arena.reset(d->budget_bytes);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the round kernel's shared memory (the inner sweep's copy stages) is above the 48 KB default
  const bool smem_ok = cudaFuncSetAttribute(serve_round_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(sizeof(SrvSmem))) == cudaSuccess;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_round_kernel, kSThreads, sizeof(SrvSmem)) !=
      cudaSuccess)
    per_sm = 1;  // one resident CTA per SM is always possible
  s->grid = std::max(1, per_sm) * sms;
  if (!smem_ok) {
    jacobi_server_destroy(s);
    return JACOBI_ERR_CUDA;
  }
  if (grow(s, 64) != JACOBI_OK || cudaMalloc(&s->d_queue, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&s->d_cols, kOzServeCols * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&s->d_tcstat, sizeof(int)) != cudaSuccess || cudaMallocHost(&s->h_tcstat, sizeof(int)) != cudaSuccess) {
    jacobi_server_destroy(s);
    return JACOBI_ERR_OUT_OF_MEMORY;
  }
  {
    int cols[kOzServeCols];
    for (int c = 0; c < kOzServeCols; ++c) cols[c] = c;
    if (cudaMemcpy(s->d_cols, cols, sizeof(cols), cudaMemcpyHostToDevice) != cudaSuccess) {
      jacobi_server_destroy(s);
      return JACOBI_ERR_CUDA;
    }
  }
  *out = s;
  return JACOBI_OK;
}

static int submit(jacobi_server* s, int64_t n, int64_t r, Request* rq, int64_t* id_out) {
  if (!s || n < 1 || n > JACOBI_SERVE_MAX_N || r < 1 || r > JACOBI_SERVE_MAX_RHS) {
    delete rq;
    return JACOBI_ERR_INVALID_ARG;
  }
  if (request_bytes(n, r, round_up(n, kLdAlign), true, s->split, s->tc) > s->arena.size) {
    delete rq;
    return JACOBI_ERR_OUT_OF_MEMORY;  // could never be admitted
  }
  rq->id = s->next_id++;
  rq->n = n;
  rq->r = r;
  s->pending.push_back(rq);
  if (id_out) *id_out = rq->id;
  return JACOBI_OK;
}

int jacobi_server_submit(jacobi_server* s, int64_t n, int64_t r, const double* A, const double* B, double* X_out,
                         int64_t* id_out) {
  if (!A || !B) return JACOBI_ERR_INVALID_ARG;
  Request* rq = new (std::nothrow) Request();
  if (!rq) return JACOBI_ERR_OUT_OF_MEMORY;
  rq->A_in = A;
  rq->B_in = B;
  rq->X_out = X_out;
  return submit(s, n, r, rq, id_out);
}

int jacobi_server_submit_generated(jacobi_server* s, int64_t n, int64_t r, double f, uint64_t seed, double* X_out,
                                   int64_t* id_out) {
  if (!(f > 0.0)) return JACOBI_ERR_INVALID_ARG;
  Request* rq = new (std::nothrow) Request();
  if (!rq) return JACOBI_ERR_OUT_OF_MEMORY;
  rq->generate = true;
  rq->f = f;
  rq->seed = seed;
  rq->X_out = X_out;
  return submit(s, n, r, rq, id_out);
}

int jacobi_server_step(jacobi_server* s, int32_t* active_out, int32_t* pending_out) {
  if (!s) return JACOBI_ERR_INVALID_ARG;
  // admit in arrival order while the budget (and the active cap) allows
  while (!s->pending.empty() && (s->max_active <= 0 || static_cast<int>(s->active.size()) < s->max_active)) {
    Request* rq = s->pending.front();
    if (!admit(s, rq)) break;
    s->pending.pop_front();
    s->active.push_back(rq);
  }
  const int na = static_cast<int>(s->active.size());
  if (na > 0) {
    if (grow(s, na) != JACOBI_OK) return JACOBI_ERR_OUT_OF_MEMORY;
    // heaviest item first: an FP64 residual item costs 16 n r_bucket FP64 FMAs, an inner-sweep or setup
    // item streams 16 n FP32 / FP64 entries (a few FP64-FMA times' worth)
    auto item_cost = [](const Request* rq) {
      const double n = static_cast<double>(rq->n);
      if (rq->q.phase == kPhResid) return n * (rq->q.split ? 0.25 : 1.0) * rq->q.rb;
      return n * (rq->q.phase == kPhPrep ? 0.5 : 0.25);
    };
    std::stable_sort(s->active.begin(), s->active.end(),
                     [&](const Request* a, const Request* b) { return item_cost(a) > item_cost(b); });
    int64_t items = 0, tiles = 0;
    int nres = 0;  // tensor-core residual requests of this round
    for (int k = 0; k < na; ++k) {
      Request* rq = s->active[static_cast<size_t>(k)];
      rq->q.st = s->d_stats + static_cast<size_t>(k) * kStatSlots;
      s->h_reqs[k] = rq->q;
      s->h_first[k] = items;
      if (s->tc && rq->q.phase == kPhResid) {
        // this request's residual runs in the grouped tensor-core launch, not in the round kernel
        OzResidParams& p = s->h_ozp[nres];
        p = OzResidParams{};
        p.n = rq->n;
        p.r = kOzServeCols;
        p.ld = rq->ld;
        p.nr = oz_padded_rows(rq->n);
        p.aexp = rq->q.aexp;
        p.xexp = rq->q.xexp;
        p.x = rq->q.X[rq->q.xsel];
        p.b = rq->q.B;
        p.d = rq->q.d;
        p.rinv = rq->q.rinv;
        p.c1 = rq->q.C1;
        p.d1 = rq->q.D[0];
        p.d1h = nullptr;
        p.colmax = rq->q.st;
        p.cols = s->d_cols;
        p.nact = rq->r;
        p.status = s->d_tcstat;
        p.wait_ns = kWaitLimitNs;
        p.xd = rq->q.xdig;
        p.xexp_w = rq->q.xexp;
        s->h_maps[2 * nres] = rq->maps[0];
        s->h_maps[2 * nres + 1] = rq->maps[1];
        s->h_ozfirst[nres] = tiles;
        tiles += p.nr / 128;
        ++nres;
      } else {
        items += (rq->n + kSRows - 1) / kSRows;
      }
    }
    s->h_first[na] = items;
    if (s->tc) s->h_ozfirst[nres] = tiles;  // the grouped arrays exist only on a tensor-core-residual server
    if (cudaMemcpyAsync(s->d_reqs, s->h_reqs, sizeof(SrvReq) * na, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(s->d_first, s->h_first, sizeof(int64_t) * (na + 1), cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(s->d_stats, 0, sizeof(unsigned long long) * kStatSlots * na, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->d_queue, 0, sizeof(unsigned long long), s->stream) != cudaSuccess)
      return JACOBI_ERR_CUDA;
    if (nres > 0) {
      if (cudaMemsetAsync(s->d_tcstat, 0, sizeof(int), s->stream) != cudaSuccess ||
          cudaMemcpyAsync(s->d_ozp, s->h_ozp, sizeof(OzResidParams) * nres, cudaMemcpyHostToDevice, s->stream) !=
              cudaSuccess ||
          cudaMemcpyAsync(s->d_maps, s->h_maps, sizeof(CUtensorMap) * 2 * nres, cudaMemcpyHostToDevice, s->stream) !=
              cudaSuccess ||
          cudaMemcpyAsync(s->d_ozfirst, s->h_ozfirst, sizeof(int64_t) * (nres + 1), cudaMemcpyHostToDevice,
                          s->stream) != cudaSuccess ||
          launch_oz_grouped(s->d_ozp, s->d_maps, s->d_ozfirst, nres, tiles, s->stream) != cudaSuccess)
        return JACOBI_ERR_CUDA;
    }
    if (items > 0) {
      const int grid = static_cast<int>(std::min<int64_t>(items, s->grid));
      serve_round_kernel<<<grid, kSThreads, sizeof(SrvSmem), s->stream>>>(s->d_reqs, na, s->d_first, items,
                                                                          s->d_queue);
      if (cudaGetLastError() != cudaSuccess) return JACOBI_ERR_CUDA;
    }
    *s->h_tcstat = 0;
    if (cudaMemcpyAsync(s->h_stats, s->d_stats, sizeof(unsigned long long) * kStatSlots * na, cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess ||
        (nres > 0 &&
         cudaMemcpyAsync(s->h_tcstat, s->d_tcstat, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
      return JACOBI_ERR_CUDA;
    if (*s->h_tcstat != 0) return JACOBI_ERR_TIMEOUT;  // a bounded wait of the residual kernel expired
    ++s->rounds;
    // move every request's state machine (Section 2 control flow per request, plus the refinement)
    std::vector<Request*> still;
    still.reserve(static_cast<size_t>(na));
    for (int k = 0; k < na; ++k) {
      Request* rq = s->active[static_cast<size_t>(k)];
      const unsigned long long* st = s->h_stats + static_cast<size_t>(k) * kStatSlots;
      SrvReq& q = rq->q;
      int finish = 1;  // 1: keep going, else the final status
      if (q.phase == kPhPrep && !rq->maps_ok) {
        finish = JACOBI_ERR_CUDA;  // the tensor maps of its digits could not be encoded
      } else if (q.phase == kPhPrep) {
        if (st[34]) {
          const unsigned long long key = ~st[34];
          finish = (key & 0xFF) == 2 ? JACOBI_ERR_ZERO_DIAGONAL : JACOBI_ERR_NONFINITE;
        } else {
          // the setup wrote C1 = B / a_ii and D0 = C1: the residual of the zero start vector is B
          rq->bnorm.assign(static_cast<size_t>(rq->r), 0.0);
          double bmax = 0.0;
          for (int64_t c = 0; c < rq->r; ++c) {
            rq->bnorm[static_cast<size_t>(c)] = as_double(st[16 + c]);
            bmax = std::max(bmax, rq->bnorm[static_cast<size_t>(c)]);
            q.xg[c] = host_split_exponent(st[40 + c]);  // the iterate's scale: max_i |b_ic / a_ii|
          }
          rq->outer = 1;
          rq->st.rel_residual = 1.0;
          if (!std::isfinite(bmax)) {
            finish = JACOBI_ERR_NONFINITE;
          } else if (bmax == 0.0) {
            rq->st.rel_residual = 0.0;
            finish = JACOBI_OK;  // B = 0: X = 0 is exact
          } else {
            q.phase = kPhInner;
            q.dsel = 0;
            rq->inner_step = 0;
          }
        }
      } else if (q.phase == kPhResid) {
        ++rq->outer;
        double rho = 0.0;
        for (int64_t c = 0; c < rq->r; ++c) {
          const double bn = rq->bnorm[static_cast<size_t>(c)];
          const double v = bn > 0.0 ? as_double(st[c]) / bn : 0.0;
          rho = (std::isnan(v) || v > rho) ? v : rho;
        }
        rq->st.rel_residual = rho;
        if (!std::isfinite(rho))
          finish = JACOBI_ERR_NONFINITE;
        else if (rho <= s->tol)
          finish = JACOBI_OK;
        else if (rq->outer >= s->max_outer || rq->inner_total >= s->max_iter)
          finish = JACOBI_NOT_CONVERGED;
        else {
          q.phase = kPhInner;
          q.dsel = 0;  // the residual round wrote D0 = C1
          rq->inner_step = 0;
        }
      } else {
        ++rq->inner_total;
        ++rq->inner_step;
        const double chg = as_double(st[32]), mag = as_double(st[33]);
        rq->st.final_delta = chg;
        q.dsel ^= 1;
        if (!std::isfinite(chg) || !std::isfinite(mag)) {
          finish = JACOBI_ERR_NONFINITE;
        } else if (chg <= static_cast<double>(s->inner_rtol) * mag || rq->inner_step >= s->max_inner ||
                   rq->inner_total >= s->max_iter) {
          q.xsel ^= 1;  // X + delta becomes the current iterate
          q.phase = kPhResid;
        }
      }
      if (finish == 1)
        still.push_back(rq);
      else
        retire(s, rq, finish);
    }
    s->active.swap(still);
  }
  if (active_out) *active_out = static_cast<int32_t>(s->active.size());
  if (pending_out) *pending_out = static_cast<int32_t>(s->pending.size());
  return JACOBI_OK;
}

int jacobi_server_poll(jacobi_server* s, int64_t* ids, jacobi_stats* stats, int32_t cap, int32_t* count) {
  if (!s || !count || cap < 0 || (cap > 0 && (!ids || !stats))) return JACOBI_ERR_INVALID_ARG;
  // results copied out by the last round are complete once the stream has caught up
  if (!s->done.empty() && cudaStreamSynchronize(s->stream) != cudaSuccess) return JACOBI_ERR_CUDA;
  const int32_t m = static_cast<int32_t>(std::min<size_t>(s->done.size(), static_cast<size_t>(cap)));
  for (int32_t i = 0; i < m; ++i) {
    ids[i] = s->done[static_cast<size_t>(i)].first;
    stats[i] = s->done[static_cast<size_t>(i)].second;
  }
  s->done.erase(s->done.begin(), s->done.begin() + m);
  *count = m;
  return JACOBI_OK;
}

int jacobi_server_wait(jacobi_server* s, int64_t id, jacobi_stats* stats) {
  if (!s || id < 1 || id >= s->next_id) return JACOBI_ERR_INVALID_ARG;
  for (;;) {
    for (auto it = s->done.begin(); it != s->done.end(); ++it)
      if (it->first == id) {
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) return JACOBI_ERR_CUDA;
        const jacobi_stats st = it->second;
        s->done.erase(it);
        if (stats) *stats = st;
        return st.status;
      }
    bool queued = false;
    for (const Request* rq : s->pending) queued = queued || rq->id == id;
    for (const Request* rq : s->active) queued = queued || rq->id == id;
    if (!queued) return JACOBI_ERR_INVALID_ARG;  // collected already by a poll or an earlier wait
    int32_t active = 0, pending = 0;
    const int st = jacobi_server_step(s, &active, &pending);
    if (st != JACOBI_OK) return st;
  }
}

int jacobi_server_rounds(jacobi_server* s, int64_t* rounds) {
  if (!s || !rounds) return JACOBI_ERR_INVALID_ARG;
  *rounds = s->rounds;
  return JACOBI_OK;
}

void jacobi_server_destroy(jacobi_server* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (Request* rq : s->pending) delete rq;
  for (Request* rq : s->active) delete rq;
  cudaFree(s->d_reqs);
  cudaFree(s->d_first);
  cudaFree(s->d_stats);
  cudaFree(s->d_queue);
  cudaFree(s->d_ozp);
  cudaFree(s->d_maps);
  cudaFree(s->d_ozfirst);
  cudaFree(s->d_cols);
  cudaFree(s->d_tcstat);
  cudaFreeHost(s->h_ozp);
  cudaFreeHost(s->h_maps);
  cudaFreeHost(s->h_ozfirst);
  cudaFreeHost(s->h_tcstat);
  cudaFreeHost(s->h_reqs);
  cudaFreeHost(s->h_first);
  cudaFreeHost(s->h_stats);
  cudaFree(s->arena_base);
  delete s;
}

int jacobi_generate_request(int64_t n, int64_t r, double f, uint64_t seed, double* A, double* B, int64_t ldb,
                            void* stream) {
  if (n < 1 || r < 1 || !A || !B || ldb < n || !(f > 0.0)) return JACOBI_ERR_INVALID_ARG;
  const int64_t blocks = std::min<int64_t>(n, 4096);
  serve_generate_kernel<<<static_cast<unsigned>(blocks), kSThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      n, r, n, ldb, f, seed, A, B);
  return cudaGetLastError() == cudaSuccess ? JACOBI_OK : JACOBI_ERR_CUDA;
}

}  // extern "C"
