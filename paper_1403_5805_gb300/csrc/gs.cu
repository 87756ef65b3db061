// Gauss-Seidel / SOR sweeps for one dense system, the relaxed relative of the Section 2 iteration:
//
//   x_i^(k) = x_i^(k-1) + omega ( (beta_i - sum_{j<i} alpha_ij x_j^(k) - sum_{j>i} alpha_ij x_j^(k-1))
//                                 / alpha_ii - x_i^(k-1) ).
//
// The sweep is sequential in i, so it is distributed as a chain over row blocks: CTA c owns rows
// [r_c, r_(c+1)).  With M = D + omega L for the block's diagonal and strict lower part, its new values are
//
//   x_c^(k) = M^-1 w,   w = (1 - omega) D x_c^(k-1) + omega (u - P x_(c-1)^(k)),
//   u = beta_c - (strict upper part of the diagonal block) x_c^(k-1) - (columns after the block) x^(k-1)
//              - (columns of blocks 0 .. c-2) x^(k),
//
// where P is the block's rows x the previous block's columns.  Splitting off the last term,
// x_c^(k) = y + Q x_(c-1)^(k) with y = M^-1 ((1 - omega) D x_c^(k-1) + omega u) and Q = -omega M^-1 P, both
// M^-1 and Q formed once per solve in shared memory.  So in sweep k CTA c
//   1. has u without the earlier blocks from the previous iteration (the strict upper part right after
//      publishing x_c^(k-1), the columns after the block as the later blocks published x^(k-1));
//   2. subtracts the columns of blocks 0 .. c-2 as each block publishes (a per-CTA flag, release / acquire);
//   3. forms y;
//   4. takes x_(c-1)^(k) from a mailbox that block c-1 fills with relaxed stores as soon as it has its values
//      (the entries start as a NaN pattern no arithmetic produces, so the data is its own flag: no fence
//      and no second round trip on the chain), empties the mailbox again, and finishes x = y + Q x_(c-1);
//   5. writes x_c^(k), fills its own mailbox, publishes its flag, and starts sweep k+1's u.
// The chain's critical path per block is one m x m shared-memory product and one L2 round trip; the streamed
// products over A from HBM and the triangular solve run while the earlier blocks hold the chain.
// The result is the sequential Gauss-Seidel / SOR sweep (up to rounding order), whatever the grid.
// Sweeps overlap: the stopping test on sweep k is read once the last block has published (no grid barrier).
// Every wait is bounded by %globaltimer; a wait that runs out sets JACOBI_ERR_TIMEOUT for the solve.
// FP64 issue is the scarce resource here (a couple of lanes per clock per SM).  So Q x and the row
// products over A run on the FP32 units as float-float (splitfloat.cuh): power-of-two scales per row of Q
// and of A and one per solve for x, integer splits into two FP32 words, error-free products; a step or
// link whose values leave the scale's range falls back to FP64.  The remaining FP64 products (M^-1 w, the
// strict upper part) split rows across two threads; reductions use halving exchanges, not per-row warp
// butterflies.
#include "device_util.cuh"
#include "gs.cuh"
#include "splitfloat.cuh"

namespace jac {
namespace {

constexpr int kGsWarps = kGsThreads / 32;

__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Mailbox entry not filled yet: a NaN pattern that no FP64 operation returns (a computed value with these
// bits, only possible by propagating such a NaN from the start vector, is stored as kNanStandIn instead).
constexpr unsigned long long kEmpty = 0xFFFFFFFFFFFFFFFFull;
constexpr unsigned long long kNanStandIn = 0x7FF8000000000001ull;

// Warp sums of sixteen per-lane values v[0..15]: lane l receives the total of v[(l >> 1) & 15].  Halving
// exchanges across lanes 16, 8, 4 and 2 apart (each lane keeps the half of its values whose row matches its
// lane bit and adds the partner's copy of them), then one across neighbouring lanes: 16 FP64 adds per warp
// for the sixteen rows, where sixteen butterflies would take 80.
__device__ __forceinline__ double warp_sum16(const double (&v)[16], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
  double a[8], b[4], d[2];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const double keep = h16 ? v[t + 8] : v[t], give = h16 ? v[t] : v[t + 8];
    a[t] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const double keep = h8 ? a[t + 4] : a[t], give = h8 ? a[t] : a[t + 4];
    b[t] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
  }
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const double keep = h4 ? b[t + 2] : b[t], give = h4 ? b[t] : b[t + 2];
    d[t] = keep + __shfl_xor_sync(0xffffffffu, give, 4);
  }
  double z = (h2 ? d[1] : d[0]) + __shfl_xor_sync(0xffffffffu, h2 ? d[0] : d[1], 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  return z;
}

// Float-float sum (two-sum of the high words, the low words added to its error, fast renormalisation).
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float hs = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(hs, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(hs, bv)), __fsub_rn(b.hi, bv));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  FF r;
  r.hi = __fadd_rn(hs, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, hs));
  return r;
}

__device__ __forceinline__ FF shfl_ff(FF v, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// warp_sum16 on float-float values (the same halving exchanges, each add a float-float sum on the FP32
// units): lane l receives the total of v[(l >> 1) & 15].
__device__ __forceinline__ FF warp_sum16_ff(const FF (&v)[16], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
  FF a[8], b[4], d[2];
#pragma unroll
  for (int t = 0; t < 8; ++t) a[t] = ff_add(h16 ? v[t + 8] : v[t], shfl_ff(h16 ? v[t] : v[t + 8], 16));
#pragma unroll
  for (int t = 0; t < 4; ++t) b[t] = ff_add(h8 ? a[t + 4] : a[t], shfl_ff(h8 ? a[t] : a[t + 4], 8));
#pragma unroll
  for (int t = 0; t < 2; ++t) d[t] = ff_add(h4 ? b[t + 2] : b[t], shfl_ff(h4 ? b[t] : b[t + 2], 4));
  FF z = ff_add(h2 ? d[1] : d[0], shfl_ff(h2 ? d[0] : d[1], 2));
  return ff_add(z, shfl_ff(z, 1));
}

// Pull the block's rows over columns [c0, c1) into L2 ahead of use (one prefetch per 128-byte line).
__device__ void prefetch_rows(const GsParams& p, int64_t r0, int m, int64_t c0, int64_t c1) {
  if (c1 <= c0) return;
  const int64_t first = c0 & ~int64_t(15), lines = (c1 - first + 15) / 16;  // 16 doubles per line
  for (int64_t e = threadIdx.x; e < m * lines; e += kGsThreads) {
    const double* q = p.A + (r0 + e / lines) * p.lda + first + (e % lines) * 16;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
  }
}

// Bounded wait until *flag >= k (thread 0 of the CTA).  False if the limit ran out or another CTA
// reported an error.
__device__ bool wait_flag(const int* flag, int k, const int* status, uint64_t limit_ns) {
  if (ld_acquire_i32(flag) >= k) return true;
  const uint64_t t0 = global_timer_ns();
  while (ld_acquire_i32(flag) < k) {
    if (ld_volatile_i32(status) < 0) return false;
    if (global_timer_ns() - t0 > limit_ns) return false;
    __nanosleep(20);
  }
  return true;
}

// Rows of A per warp in the row products (8 warps cover the largest block).
constexpr int kGsRowsPerWarp = (kGsMaxRows + kGsWarps - 1) / kGsWarps;
static_assert(kGsRowsPerWarp <= 16, "the row sums are reduced sixteen at a time");

// One step of the row products: kCols columns per lane (j0 + lane + 32 t, t < kCols; those at or past c1
// predicated off), every load issued before the arithmetic.  The products run on the FP32 units as
// float-float: a_ij scaled by 2^-re_i (re_i: split exponent of the row maximum) and x_j by 2^-g, each split
// with integer operations into its top 24 and next 23 significant bits, the error of hi * hi recovered by
// an FMA (splitfloat.cuh).  A step whose x values reach 2^(g + 100) (or are not finite) runs in FP64
// instead and is reduced into u at once.
template <int kCols>
__device__ __forceinline__ void rows_step(const double* a, int64_t lda, int nr, int64_t j0, int64_t c1, const double* x,
                                          FF (&acc)[16], const int* re, int g, double* u, int lane) {
  double xv[kCols], av[kCols][kGsRowsPerWarp];
#pragma unroll
  for (int t = 0; t < kCols; ++t) {
    const int64_t j = j0 + lane + 32 * t;
    const bool ok = j < c1;
    xv[t] = ok ? __ldcg(x + j) : 0.0;
#pragma unroll
    for (int q = 0; q < kGsRowsPerWarp; ++q) av[t][q] = ok && q < nr ? __ldg(a + q * lda + j) : 0.0;
  }
  bool bad = false;
#pragma unroll
  for (int t = 0; t < kCols; ++t) {
    const int be = (static_cast<uint32_t>(__double2hiint(xv[t])) >> 20) & 0x7FF;
    bad |= be == 0x7FF || be - 1023 >= g + 100;
  }
  if (!__any_sync(0xffffffffu, bad)) {
    float xh[kCols], xl[kCols];
#pragma unroll
    for (int t = 0; t < kCols; ++t) split_scaled(xv[t], g, xh[t], xl[t]);
#pragma unroll
    for (int q = 0; q < kGsRowsPerWarp; ++q)
      if (q < nr) {
        const int sh = re[q];
#pragma unroll
        for (int t = 0; t < kCols; ++t) {
          float ah, al;
          split_scaled(av[t][q], sh, ah, al);
          ff_fma(acc[q], ah, al, xh[t], xl[t]);
        }
        ff_renorm(acc[q]);
      }
  } else {
    double part[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) part[q] = 0.0;
#pragma unroll
    for (int t = 0; t < kCols; ++t)
#pragma unroll
      for (int q = 0; q < kGsRowsPerWarp; ++q)
        if (q < nr) part[q] = fma(av[t][q], xv[t], part[q]);
    const double sum = warp_sum16(part, lane);
    const int q = (lane >> 1) & 15;
    if ((lane & 1) == 0 && q < nr) u[q] -= sum;
  }
}

// Row products over A for the warp's rows i0 .. i0+nr-1 (nr <= kGsRowsPerWarp): acc[q] += a_(r0+i0+q),j x_j
// over the lane's columns j = c0 + lane + 32 t in [c0, c1).  Lanes read 32 consecutive columns of a row
// (coalesced), up to 128 columns per step with every load of the step issued before its arithmetic; the
// steps are the same for all lanes (the ragged end is predicated) and the last one is only as wide as the
// columns left, so a block costs one memory latency and few idle lanes.  The per-lane float-float sums
// stay in registers across calls and are reduced once per phase (flush_rows).  x is read through L2
// (other CTAs write it during the launch).  re: the warp's rows' scale exponents; u: the warp's rows of u.
__device__ __forceinline__ void rows_dot(const GsParams& p, int64_t r0, int i0, int nr, int64_t c0, int64_t c1,
                                         const double* x, FF (&acc)[16], const int* re, int g, double* u, int lane) {
  if (nr <= 0) return;
  const double* a = p.A + (r0 + i0) * p.lda;
  int64_t j0 = c0;
  for (; c1 - j0 > 96; j0 += 128) rows_step<4>(a, p.lda, nr, j0, c1, x, acc, re, g, u, lane);
  const int64_t rem = c1 - j0;
  if (rem > 64)
    rows_step<3>(a, p.lda, nr, j0, c1, x, acc, re, g, u, lane);
  else if (rem > 32)
    rows_step<2>(a, p.lda, nr, j0, c1, x, acc, re, g, u, lane);
  else if (rem > 0)
    rows_step<1>(a, p.lda, nr, j0, c1, x, acc, re, g, u, lane);
}

// u[q] -= the warp's float-float sums of acc[q] (q < nr), back in FP64 at scale 2^(re_q + g); acc cleared.
__device__ __forceinline__ void flush_rows(FF (&acc)[16], double* u, const int* re, int g, int nr, int lane) {
  if (nr <= 0) return;
  const FF t = warp_sum16_ff(acc, lane);
  const int q = (lane >> 1) & 15;
  if ((lane & 1) == 0 && q < nr)
    u[q] -= (static_cast<double>(t.hi) + static_cast<double>(t.lo)) * pow2(re[q]) * pow2(g);
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = FF{0.0f, 0.0f};
}

// acc (and u) -= the columns of blocks [b0, b1) with x for the warp's rows, taking each block once its flag reaches kf
// (in block order, runs of already-published blocks at once), and pulling the next awaited block into L2
// meanwhile.  Called by the whole CTA.  A wait that runs out clears *s_ok and skips the rest.
__device__ void process_published(const GsParams& p, int64_t r0, int m, int i0, int nr, int b0, int b1, int kf,
                                  const double* x, FF (&acc)[16], const int* re, int g, double* u, int lane, int* s_e,
                                  int* s_ok) {
  const int G = gridDim.x;
  if (b0 < b1) prefetch_rows(p, r0, m, p.n * b0 / G, p.n * (b0 + 1) / G);
  int done = b0;
  while (done < b1) {
    __syncthreads();
    if (threadIdx.x == 0) {
      int e;
      if (*s_ok && wait_flag(p.flags + done, kf, &p.ctl->status, p.wait_ns)) {
        e = done + 1;
        while (e < b1 && ld_acquire_i32(p.flags + e) >= kf) ++e;
      } else {
        *s_ok = 0;
        e = b1;
      }
      *s_e = e;
    }
    __syncthreads();
    const int e = *s_e;
    if (e < b1) prefetch_rows(p, r0, m, p.n * e / G, p.n * (e + 1) / G);
    if (*s_ok) rows_dot(p, r0, i0, nr, p.n * done / G, p.n * e / G, x, acc, re, g, u, lane);
    done = e;
  }
}

__device__ __forceinline__ double bits_to_double(unsigned long long v) {
  return __longlong_as_double(static_cast<long long>(v));
}

__global__ void __launch_bounds__(kGsThreads, 1) gs_solve_kernel(GsParams p) {
  extern __shared__ double sm[];
  constexpr int P = kGsPitch;
  double* dm = sm;                    // lower with diagonal: (M^-1)_ij; strict upper: a_(r0+i),(r0+j)
  double* qm = dm + kGsMaxRows * P;   // Q = -omega M^-1 P, P_ij = a_(r0+i),(s+j) (the previous block's columns)
  double* xo_b = qm + kGsMaxRows * P; // x^(k-1) of the block
  double* u = xo_b + kGsMaxRows;      // running right-hand side of the block's rows
  double* w = u + kGsMaxRows;         // (1 - omega) D x^(k-1) + omega u
  double* xn_b = w + kGsMaxRows;      // x^(k) of the block
  double* xp = xn_b + kGsMaxRows;     // x^(k) of the previous block
  float2* xpf = reinterpret_cast<float2*>(xp + kGsMaxRows);  // the same as float-float pairs at scale 2^-g
  int* qe = reinterpret_cast<int*>(xpf + kGsMaxRows);        // row scale exponents of Q
  int* rex = qe + kGsMaxRows;                                 // row scale exponents of A
  float2* qf = reinterpret_cast<float2*>(qm);                 // Q as float-float pairs (in place, after setup)
  __shared__ unsigned long long s_red[kGsWarps];
  __shared__ double s_sq[kGsWarps];
  __shared__ int s_e, s_ok, s_next, s_status;

  const int G = gridDim.x, c = blockIdx.x;
  const int64_t r0 = p.n * c / G, r1 = p.n * (c + 1) / G;
  const int64_t sp = c > 0 ? p.n * (c - 1) / G : 0;  // first column of the previous block
  const int m = static_cast<int>(r1 - r0), mp = static_cast<int>(r0 - sp);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the block products run two threads per row (row ri, even or odd columns), on whole warps
  const int ri = tid >> 1, par = tid & 1;
  const bool row_ok = ri < m;
  // the row products over A: warp w takes rows [w rpw, (w + 1) rpw)
  const int rpw = (m + kGsWarps - 1) / kGsWarps;
  const int i0 = warp * rpw, nr = max(0, min(rpw, m - i0));
  FF acc[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) acc[t] = FF{0.0f, 0.0f};
  const double om = p.omega;
  if (tid == 0 && c == 0) p.ctl->t_start = global_timer_ns();

  // ---- once per solve: M^-1 for M = D + omega L of the diagonal block (staged in qm first), the block's
  // strict upper part, then Q from the previous block's columns
  for (int e = tid; e < m * m; e += kGsThreads) {
    const int i = e / m, j = e % m;
    qm[i * P + j] = p.A[(r0 + i) * p.lda + r0 + j];
  }
  __syncthreads();
  if (tid < m) {
    // column t by forward substitution: z_t = 1 / a_tt, z_i = -(sum_{t<=j<i} omega a_ij z_j) / a_ii
    const int t = tid;
    dm[t * P + t] = __ldg(p.rinv + r0 + t);
    for (int i = t + 1; i < m; ++i) {
      double s = 0.0;
      for (int j = t; j < i; ++j) s = fma(qm[i * P + j], dm[j * P + t], s);
      dm[i * P + t] = -(om * s) * __ldg(p.rinv + r0 + i);
    }
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += kGsThreads) {
    const int i = e / m, j = e % m;
    if (j > i) dm[i * P + j] = qm[i * P + j];
  }
  __syncthreads();
  for (int e = tid; e < m * mp; e += kGsThreads) {
    const int i = e / mp, j = e % mp;
    qm[i * P + j] = p.A[(r0 + i) * p.lda + sp + j];
  }
  __syncthreads();
  if (c > 0 && tid < 2 * kGsMaxRows) {
    // in place, a pair of threads per column, bottom-up: row i of Q needs rows <= i of P only
    const int j = tid >> 1;
    const bool col_ok = j < mp;
    for (int i = m - 1; i >= 0; --i) {
      double s = 0.0;
      if (col_ok)
        for (int t = par; t <= i; t += 2) s = fma(dm[i * P + t], qm[t * P + j], s);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      if (col_ok && par == 0) qm[i * P + j] = -om * s;
    }
  }
  __syncthreads();
  // Q as float-float pairs: row i scaled by 2^-qe_i (qe_i the split exponent of max_j |Q_ij|), each entry
  // split with integer operations into its top 24 and next 23 significant bits, in place
  if (c > 0) {
    if (tid < m) {
      uint32_t mb = 0;
      for (int j = 0; j < mp; ++j) {
        const uint32_t h = abs_hi(qm[tid * P + j]);
        mb = h > mb ? h : mb;
      }
      qe[tid] = split_exponent_hi(mb);
    }
    __syncthreads();
    for (int e = tid; e < m * mp; e += kGsThreads) {
      const int i = e / mp, j = e % mp;
      float h, l;
      split_scaled(qm[i * P + j], qe[i], h, l);
      qf[i * P + j] = make_float2(h, l);
    }
    __syncthreads();
  }
  // the scale of the float-float split of the previous block's values: x^(k) stays within a modest factor
  // of max_i |b_i / a_ii| for a convergent iteration; a link whose values reach 2^(g + 100) (or are not
  // finite) runs in FP64 instead
  const int g = split_exponent(__ldg(p.cmax));
  for (int i = tid; i < m; i += kGsThreads) rex[i] = __ldg(p.rexp + r0 + i);

  // u_i = beta_i - sum_{j > i in the block} a_ij x_j with the block's own values xs (all threads call it)
  auto start_u = [&](const double* xs) {
    double s = 0.0;
    if (row_ok)
      for (int j = ri + 1 + par; j < m; j += 2) s = fma(dm[ri * P + j], xs[j], s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (row_ok && par == 0) u[ri] = __ldg(p.b + r0 + ri) - s;
  };

  // ---- sweeps.  Iteration k ends with this block's x^(k) published, then already computes the part of
  // sweep k+1 that needs the previous iterate (the strict upper part, and the columns after the block from
  // x^(k) of the later blocks, taken as they publish), and decides on sweep k once the last block has
  // published it: every block's change norm is in red[k % 3] / part by then (each block adds its own before
  // publishing, and the flags are released and acquired in chain order), so every CTA takes the same
  // decision with no grid barrier, and the next sweep's chain starts as soon as the last block of this one
  // is done.  x^(k) lives in xb for odd k, xa for even k; x^(0) (the start vector) in xa.  The mailbox of
  // block c for sweep k is mbox[(k & 1) n + r_c ...].
  int64_t k = 1;
  double delta = 0.0;
  int status = kStatusNotConverged;
  if (tid == 0) s_ok = 1;
  for (int i = tid; i < m; i += kGsThreads) xo_b[i] = __ldcg(p.xa + r0 + i);
  __syncthreads();
  start_u(xo_b);
  __syncthreads();
  rows_dot(p, r0, i0, nr, r1, p.n, p.xa, acc, rex + i0, g, u + i0, lane);  // sweep 1: the later blocks' x^(0)
  flush_rows(acc, u + i0, rex + i0, g, nr, lane);
  for (;; ++k) {
    double* xn = (k & 1) ? p.xb : p.xa;
    unsigned long long* box = p.mbox + (k & 1) * p.n;
    // the blocks before the previous one, with x^(k), as they are published (in order)
    process_published(p, r0, m, i0, nr, 0, c - 1, static_cast<int>(k), xn, acc, rex + i0, g, u + i0, lane, &s_e,
                      &s_ok);
    flush_rows(acc, u + i0, rex + i0, g, nr, lane);
    __syncthreads();
    for (int i = tid; i < m; i += kGsThreads)
      w[i] = om == 1.0 ? u[i] : fma(1.0 - om, __ldg(p.d + r0 + i) * xo_b[i], om * u[i]);
    __syncthreads();
    // y = M^-1 w
    double x = 0.0;
    if (row_ok)
      for (int j = par; j <= ri; j += 2) x = fma(dm[ri * P + j], w[j], x);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    if (c > 0) {
      // x_(c-1)^(k) from the previous block's mailbox, one entry per thread, emptied again for sweep k+2
      int bad = 0;
      if (tid < mp) {
        unsigned long long* e = box + sp + tid;
        unsigned long long v = ld_relaxed_u64(e);
        if (v == kEmpty && s_ok) {
          const uint64_t t0 = global_timer_ns();
          while ((v = ld_relaxed_u64(e)) == kEmpty) {
            if (global_timer_ns() - t0 > p.wait_ns) {
              s_ok = 0;
              break;
            }
          }
        }
        const double xv = __longlong_as_double(static_cast<long long>(v));
        xp[tid] = xv;
        const int be = static_cast<int>((v >> 52) & 0x7FFu);
        bad = be == 0x7FF || be - 1023 >= g + 100;
        float h, l;
        split_scaled(xv, g, h, l);
        xpf[tid] = make_float2(h, l);
        st_relaxed_u64(e, kEmpty);
      }
      const int any_bad = __syncthreads_or(bad);
      // x = y + Q x_(c-1): on the FP32 units as float-float products (renormalised every 8), the pair's two
      // halves summed in FP64 and scaled back by 2^(qe_i + g); FP64 when a value is out of range
      double s = 0.0;
      if (!any_bad) {
        FF a{0.0f, 0.0f};
        if (row_ok)
          for (int j = par, cnt = 1; j < mp; j += 2, ++cnt) {
            const float2 q = qf[ri * P + j], xv = xpf[j];
            ff_fma(a, q.x, q.y, xv.x, xv.y);
            if ((cnt & 7) == 0) ff_renorm(a);
          }
        double d = static_cast<double>(a.hi) + static_cast<double>(a.lo);
        d += __shfl_xor_sync(0xffffffffu, d, 1);
        if (row_ok) s = d * pow2(qe[ri]) * pow2(g);
      } else {
        if (row_ok) {
          const double sc = pow2(qe[ri]);
          for (int j = par; j < mp; j += 2) {
            const float2 q = qf[ri * P + j];
            s = fma((static_cast<double>(q.x) + static_cast<double>(q.y)) * sc, xp[j], s);
          }
        }
        s += __shfl_xor_sync(0xffffffffu, s, 1);
      }
      x += s;
    }
    unsigned long long mx = 0;
    double sq = 0.0;
    const bool withhold = p.test_skip_publish && c == 0 && k == 1;  // test hook: the chain never starts
    if (row_ok && par == 0) {
      if (c + 1 < G && !withhold) {  // the next block's input first
        const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
        st_relaxed_u64(box + r0 + ri, bits == kEmpty ? kNanStandIn : bits);
      }
      xn_b[ri] = x;
      xn[r0 + ri] = x;
      const double diff = x - xo_b[ri];
      mx = abs_bits(diff);
      if (p.norm == JACOBI_NORM_2) sq = diff * diff;
    }
    // the block's change norm, then x^(k) published
    mx = warp_max_u64(mx);
    if (p.norm == JACOBI_NORM_2) sq = warp_sum(sq);
    if (lane == 0) {
      s_red[warp] = mx;
      s_sq[warp] = sq;
    }
    __syncthreads();
    const int slot = static_cast<int>(k % 3);
    if (tid == 0) {
      unsigned long long bm = 0;
      double bs = 0.0;
      for (int q = 0; q < kGsWarps; ++q) bm = s_red[q] > bm ? s_red[q] : bm;
      if (p.norm == JACOBI_NORM_2)
        for (int q = 0; q < kGsWarps; ++q) bs += s_sq[q];  // fixed order
      if (c == 0) p.ctl->red[slot][0] = 0ull;  // the first block of the sweep opens its slot
      if (p.norm == JACOBI_NORM_2)
        p.part[slot * kMaxGrid + c] = bs;
      else if (bm)
        atomicMax(&p.ctl->red[slot][0], bm);
      if (withhold) s_ok = 0;
      if (!s_ok) atomicMin(&p.ctl->status, kStatusTimeout);
      __threadfence();
      if (!withhold) st_release_i32(p.flags + c, static_cast<int>(k));
    }
    // sweep k+1: the strict upper part with x^(k) of the block, then the columns after the block from x^(k)
    // of the later blocks as they publish
    for (int i = tid; i < m; i += kGsThreads) xo_b[i] = xn_b[i];
    start_u(xn_b);
    __syncthreads();
    process_published(p, r0, m, i0, nr, c + 1, G, static_cast<int>(k), xn, acc, rex + i0, g, u + i0, lane, &s_e,
                      &s_ok);
    flush_rows(acc, u + i0, rex + i0, g, nr, lane);
    // decision on sweep k: the last block has published it (waited for above, or this is the last block)
    __syncthreads();
    if (tid == 0) {
      double dk;
      if (p.norm == JACOBI_NORM_2) {
        double acc = 0.0;
        for (int j = 0; j < G; ++j) acc += __ldcg(p.part + slot * kMaxGrid + j);
        dk = sqrt(acc);
      } else {
        dk = bits_to_double(__ldcg(&p.ctl->red[slot][0]));
      }
      if (c == 0 && k - 1 < kTraceCap) {
        p.ctl->t_end[k - 1] = global_timer_ns();
        p.ctl->kind[k - 1] = JACOBI_PHASE_SWEEP64;
        p.ctl->nphase = static_cast<int>(k);
      }
      int next = 0;
      if (!s_ok || ld_volatile_i32(&p.ctl->status) < 0) {
        status = kStatusTimeout;
        next = 1;
      } else if (!isfinite(dk)) {
        status = kStatusNonfinite;
        next = 1;
      } else if (dk < p.tol) {
        status = kStatusOk;
        next = 1;
      } else if (k >= p.max_iter) {
        status = kStatusNotConverged;
        next = 1;
      }
      delta = dk;
      s_next = next;
      s_status = status;
    }
    __syncthreads();
    if (s_next) break;
  }
  // x^(k) of the block
  status = s_status;
  if (status != kStatusTimeout)
    for (int i = tid; i < m; i += kGsThreads) p.x_out[r0 + i] = xn_b[i];
  if (c == 0 && tid == 0) {
    jacobi_stats st;
    st.sweeps = k;
    st.outer_steps = 0;
    st.final_delta = delta;
    st.rel_residual = __longlong_as_double(0x7FF8000000000000ll);
    st.status = status;
    st.converged = status == kStatusOk;
    p.ctl->result = st;
    if (p.stats_out) *p.stats_out = st;
  }
}

}  // namespace

cudaError_t launch_gs_solve(const GsParams& p, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(gs_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kGsSmem));
  if (e != cudaSuccess) return e;
  GsParams copy = p;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(gs_solve_kernel), dim3(grid), dim3(kGsThreads),
                                     args, kGsSmem, s);
}

namespace {
// rexp[i] = split exponent of max_j |a_ij| (one CTA per row; 32-bit running maximum of the high words)
__global__ void gs_row_exponent_kernel(const double* __restrict__ A, int64_t lda, int64_t n, int* rexp) {
  const int64_t i = blockIdx.x;
  const double* row = A + i * lda;
  uint32_t mb = 0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const uint32_t h = abs_hi(__ldcs(row + j));
    mb = h > mb ? h : mb;
  }
  mb = __reduce_max_sync(0xffffffffu, mb);
  __shared__ uint32_t s_mb[8];
  if ((threadIdx.x & 31) == 0) s_mb[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) mb = s_mb[w] > mb ? s_mb[w] : mb;
    mb = s_mb[0] > mb ? s_mb[0] : mb;
    rexp[i] = split_exponent_hi(mb);
  }
}
}  // namespace

cudaError_t launch_gs_row_exponents(const double* A, int64_t lda, int64_t n, int* rexp, cudaStream_t s) {
  gs_row_exponent_kernel<<<static_cast<unsigned>(n), 256, 0, s>>>(A, lda, n, rexp);
  return cudaGetLastError();
}

int gs_max_grid() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(gs_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kGsSmem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gs_solve_kernel, kGsThreads, kGsSmem) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

}  // namespace jac
