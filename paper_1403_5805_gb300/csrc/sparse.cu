// Sparse Jacobi sweeps: the Section 2 component update with the sum over the stored entries of row i,
//
//   x_i^(k) = ( beta_i - sum_{stored j != i} alpha_ij x_j^(k-1) ) / alpha_ii,
//
// for the banded and PDE-shaped matrices of the Jacobi codes for differential equations that the paper's
// related work cites.  Setup forms the fixed-point form of Section 2, T = D^-1 (L + U) and C = D^-1 B,
// i.e. t_ij = -a_ij / a_ii and c_i = b_i / a_ii (IEEE divisions), and keeps T as a sliced-ELL copy:
// slices of 32 rows, one warp per slice and one row per lane, each slice as wide as its longest row and
// stored column-major, so that the warp's loads of the t-th entries of its 32 rows are one contiguous
// 256-byte run.  A sweep is then x_i = c_i + sum_j t_ij x_j: a row of w stored entries costs w FP64 FMAs
// plus one subtraction for the change, which matters on GB300, whose FP64 issue rate (about 2 per clock
// per SM) would otherwise bound these short rows as tightly as HBM does.  A row's entries keep their
// ascending column order, so the sum runs in the same order as the oracle's.
//
// One persistent cooperative launch runs the whole solve: per sweep each warp streams its slices (values
// and columns with the evict-first hint, so the iterate stays in L2 for the gathers), writes x^(k) and
// keeps the change norm; the norm is combined over the grid (an order-free max of IEEE bits, or fixed-order
// per-CTA partial sums for the Euclidean norm) at the one grid barrier of the sweep, and every CTA takes
// the same stop decision.  Every wait is bounded by %globaltimer and reports JACOBI_ERR_TIMEOUT.
#include <cuda_bf16.h>

#include <algorithm>
#include <initializer_list>
#include <type_traits>

#include "device_util.cuh"
#include "sparse.cuh"

namespace jac {
namespace {

constexpr int kCsrThreads = 768;
constexpr int kCsrMinBlocks = 2;  // 48 warps per SM, up to 42 registers each
constexpr int kCsrWarps = kCsrThreads / 32;

__global__ void csr_check_kernel(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ val, double* d, int32_t* lens, unsigned long long* key) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e0 = rp[i], e1 = rp[i + 1];
  const unsigned long long row = static_cast<unsigned long long>(i) << 8;
  unsigned long long bad = ~0ull;
  if (e0 < 0 || e1 < e0 || e1 > nnz || (i == 0 && e0 != 0)) {
    bad = row | 1u;
  } else {
    double dv = 0.0;
    int32_t prev = -1, cnt = 0;
    for (int64_t e = e0; e < e1; ++e) {
      const int32_t c = ci[e];
      if (c < 0 || c >= n || c <= prev) {
        bad = row | 1u;
        break;
      }
      prev = c;
      if (c == i)
        dv = val[e];
      else
        ++cnt;
    }
    if (bad == ~0ull) {
      if (!isfinite(dv)) {
        bad = (1ull << 56) | row | 3u;
      } else if (dv == 0.0) {
        bad = (1ull << 56) | row | 2u;
      } else {
        d[i] = dv;
        lens[i] = cnt;
      }
    }
  }
  if (bad != ~0ull) atomicMin(key, bad);
}

__global__ void csr_widths_kernel(int64_t n, int64_t nslices, const int32_t* __restrict__ lens, int32_t* width) {
  const int64_t s = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nslices) return;  // whole warps: nslices is a count of warps
  const int64_t i = s * kSliceRows + lane;
  const int32_t w = __reduce_max_sync(0xffffffffu, i < n ? lens[i] : 0);
  if (lane == 0) width[s] = w;
}

__global__ void csr_fill_kernel(int64_t n, int64_t nslices, const int64_t* __restrict__ rp,
                                const int32_t* __restrict__ ci, const double* __restrict__ val,
                                const double* __restrict__ d, const int64_t* __restrict__ soff, double* sval,
                                int32_t* scol, double* c, unsigned long long* bmax) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t s = i / kSliceRows;
  if (s >= nslices) return;
  const int lane = static_cast<int>(i % kSliceRows);
  const int64_t base = soff[s] + lane, w = (soff[s + 1] - soff[s]) / kSliceRows;
  int64_t t = 0;
  if (i < n) {
    const double di = d[i];
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int32_t col = ci[e];
      if (col == i) continue;
      sval[base + kSliceRows * t] = -val[e] / di;  // t_ij = -a_ij / a_ii
      scol[base + kSliceRows * t] = col;
      ++t;
    }
    const double bi = c[i];
    atomicMax(bmax, abs_bits(bi));
    c[i] = bi / di;  // c_i = b_i / a_ii (c holds b on entry)
  }
  const int32_t self = static_cast<int32_t>(i < n ? i : n - 1);
  for (; t < w; ++t) {
    sval[base + kSliceRows * t] = 0.0;
    scol[base + kSliceRows * t] = self;
  }
}

// DIA setup: every off-diagonal entry's offset j - i must be one of doff[0..ndiag) (else *bad = 1).
__global__ void csr_dia_check_kernel(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const int32_t* __restrict__ doff, int ndiag, int* bad) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
    const int64_t off = static_cast<int64_t>(ci[e]) - i;
    if (off == 0) continue;
    bool found = false;
    for (int t = 0; t < ndiag; ++t) found = found || doff[t] == off;
    if (!found) {
      atomicOr(bad, 1);
      return;
    }
  }
}

// DIA setup: entry t of row i, -a_ij / a_ii for j = i + doff[t], at ((i / 32) * ndiag + t) * 32 + i % 32
// (dval zeroed beforehand); c_i = b_i / a_ii (c holds b on entry); *bmax receives the IEEE bits of
// ||b||_inf.
__global__ void csr_dia_fill_kernel(int64_t n, const int64_t* __restrict__ rp,
                                    const int32_t* __restrict__ ci, const double* __restrict__ val,
                                    const double* __restrict__ d, const int32_t* __restrict__ doff, int ndiag,
                                    double* dval, double* c, unsigned long long* bmax) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double di = d[i];
  for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
    const int64_t off = static_cast<int64_t>(ci[e]) - i;
    if (off == 0) continue;
    for (int t = 0; t < ndiag; ++t)
      if (doff[t] == off)  // t_ij = -a_ij / a_ii
        dval[((i / kSliceRows) * ndiag + t) * kSliceRows + i % kSliceRows] = -val[e] / di;
  }
  const double bi = c[i];
  atomicMax(bmax, abs_bits(bi));
  c[i] = bi / di;
}

__device__ __forceinline__ double bits_to_double(unsigned long long v) {
  return __longlong_as_double(static_cast<long long>(v));
}

// Storage formats of T, as accessors of a slice's entries.  Sliced ELL: slice s holds w_s slots per row
// at soff[s] + 32 t + lane with explicit columns.  Diagonal (DIA): every row has the same ndiag offsets
// doff[0] < ... < doff[ndiag-1] (j = i + doff[t]; absent entries are zero), entry t of row 32 s + lane at
// (s * ndiag + t) * 32 + lane (a slice's diagonals contiguous, as an ELL slice of width ndiag), and no
// column array at all; the gathered vectors carry a zero halo of max |doff| entries on both sides, so
// i + doff[t] is always a valid index.  In both formats a row's entries run in ascending column order.
struct EllFmt {
  __device__ static int width(const CsrParams& p, int64_t s, int64_t& o0) {
    o0 = __ldg(p.soff + s);
    return static_cast<int>((__ldg(p.soff + s + 1) - o0) / kSliceRows);
  }
  __device__ static int64_t at(const CsrParams&, int64_t o0, int t, int lane) { return o0 + lane + kSliceRows * t; }
  __device__ static int64_t col(const CsrParams& p, int64_t o0, int t, int lane, int64_t, const int*) {
    return __ldcs(p.scol + o0 + lane + kSliceRows * t);
  }
  // pull slice s's values and columns into L2, one 128-byte line per lane
  __device__ static void prefetch(const CsrParams& p, int64_t s, int lane) {
    const int64_t q0 = __ldg(p.soff + s), q1 = __ldg(p.soff + s + 1);
    const int64_t vl = (q1 - q0) / 16, cl = (q1 - q0) / 32;  // lines of values (8 B) and columns (4 B)
    for (int64_t l = lane; l < vl + cl; l += 32) {
      const char* a = l < vl ? reinterpret_cast<const char*>(p.sval + q0) + 128 * l
                             : reinterpret_cast<const char*>(p.scol + q0) + 128 * (l - vl);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
  }
};
struct DiaFmt {
  __device__ static int width(const CsrParams& p, int64_t s, int64_t& o0) {
    o0 = s * p.ndiag * kSliceRows;
    return p.ndiag;
  }
  __device__ static int64_t at(const CsrParams&, int64_t o0, int t, int lane) { return o0 + lane + kSliceRows * t; }
  __device__ static int64_t col(const CsrParams&, int64_t, int t, int, int64_t i, const int* sdoff) {
    return i + sdoff[t];
  }
  __device__ static void prefetch(const CsrParams& p, int64_t s, int lane) {
    if (lane < 2 * p.ndiag)  // the slice's values: two 128-byte lines of FP64 per diagonal
      asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(p.sval + s * p.ndiag * kSliceRows) +
                                                    128 * lane));
  }
};

// The offsets of a DIA matrix in shared memory (every thread of the CTA calls it once).
__device__ __forceinline__ void load_doff(const CsrParams& p, int* sdoff) {
  if (threadIdx.x < kMaxDiag) sdoff[threadIdx.x] = threadIdx.x < p.ndiag ? p.doff[threadIdx.x] : 0;
  __syncthreads();
}

// kResid: the change norm is max |a_ii (x^(k) - x^(k-1))| / ||b||_inf (JACOBI_NORM_RESID), a separate
// instantiation so that the other norms' loop carries no extra load.
template <bool kResid, class F>
__global__ void __launch_bounds__(kCsrThreads, kCsrMinBlocks) csr_solve_kernel(CsrParams p) {
  __shared__ unsigned long long s_mx[kCsrWarps];
  __shared__ double s_sq[kCsrWarps];
  __shared__ int s_next, s_status;
  __shared__ double s_delta;
  __shared__ int sdoff[kMaxDiag];
  load_doff(p, sdoff);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * kCsrWarps + warp;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kCsrWarps;
  const int G = gridDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) p.ctl->t_start = global_timer_ns();

  int64_t k = 1;
  for (;; ++k) {
    const double* xc = (k & 1) ? p.xa : p.xb;  // x^(k-1)
    double* xn = (k & 1) ? p.xb : p.xa;        // x^(k)
    unsigned long long mx = 0;
    double sq = 0.0;
    for (int64_t s = gw; s < p.nslices; s += nw) {
      int64_t o0;
      const int w = F::width(p, s, o0);
      // pull the warp's next slice into L2 meanwhile
      if (s + nw < p.nslices) F::prefetch(p, s + nw, lane);
      const int64_t i = s * kSliceRows + lane;
      const bool live = i < p.n;
      const double xo = live ? __ldcg(xc + i) : 0.0;
      double x = live ? __ldcs(p.c + i) : 0.0;
#pragma unroll 4
      for (int t = 0; t < w; ++t)
        x = fma(__ldcs(p.sval + F::at(p, o0, t, lane)), __ldcg(xc + F::col(p, o0, t, lane, i, sdoff)), x);
      if (live) {
        const double diff = x - xo;
        xn[i] = x;
        const unsigned long long bb = abs_bits(kResid ? __ldg(p.d + i) * diff : diff);
        mx = bb > mx ? bb : mx;
        if (p.norm == JACOBI_NORM_2) sq = fma(diff, diff, sq);
      }
    }
    mx = warp_max_u64(mx);
    if (p.norm == JACOBI_NORM_2) sq = warp_sum(sq);
    if (lane == 0) {
      s_mx[warp] = mx;
      s_sq[warp] = sq;
    }
    __syncthreads();
    if (warp == 0) {
      const uint32_t phase = static_cast<uint32_t>(k - 1);
      const int slot = static_cast<int>(phase % 3);
      int ok = 1;
      if (lane == 0) {
        unsigned long long bm = 0;
        double bs = 0.0;
        for (int q = 0; q < kCsrWarps; ++q) bm = s_mx[q] > bm ? s_mx[q] : bm;
        if (p.norm == JACOBI_NORM_2) {
          for (int q = 0; q < kCsrWarps; ++q) bs += s_sq[q];  // fixed order
          p.part[(k & 1) * kMaxGrid + blockIdx.x] = bs;
        } else if (bm) {
          atomicMax(&p.ctl->red[slot][0], bm);
        }
        if (blockIdx.x == 0) p.ctl->red[(phase + 1) % 3][0] = 0ull;  // opened before anyone passes the barrier
        if (p.test_skip_arrival && blockIdx.x == 0 && phase == 0) {
          ok = 0;
          atomicMin(&p.ctl->status, kStatusTimeout);  // the others leave their wait on the error word
        } else {
          ok = grid_arrive_and_wait(&p.ctl->arrive, &p.ctl->status, (phase + 1) * static_cast<uint32_t>(G),
                                    p.wait_ns);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();  // the other lanes read after lane 0's acquire of the grid barrier
      double dk;
      if (p.norm == JACOBI_NORM_2) {
        double acc = 0.0;
        for (int j = lane; j < G; j += 32) acc += __ldcg(p.part + (k & 1) * kMaxGrid + j);
        dk = sqrt(warp_sum(acc));
      } else {
        dk = bits_to_double(__ldcg(&p.ctl->red[slot][0]));
        if (kResid) dk = dk / p.bnorm;  // ||b - A x^(k-1)|| / ||b||, as the oracle
      }
      if (lane == 0) {
        if (blockIdx.x == 0 && phase < static_cast<uint32_t>(kTraceCap)) {
          p.ctl->t_end[phase] = global_timer_ns();
          p.ctl->kind[phase] = JACOBI_PHASE_SWEEP64;
          p.ctl->nphase = static_cast<int>(phase) + 1;
        }
        int next = 1, status = kStatusNotConverged;
        if (!ok) {
          status = kStatusTimeout;
          atomicMin(&p.ctl->status, kStatusTimeout);
        } else if (!isfinite(dk)) {
          status = kStatusNonfinite;
        } else if (dk < p.tol) {
          status = kStatusOk;
        } else if (k < p.max_iter) {
          next = 0;
        }
        s_next = next;
        s_status = status;
        s_delta = dk;
      }
    }
    __syncthreads();
    if (s_next) break;
  }
  // the newest iterate is the result: converged, capped (X^(L)) or non-finite alike
  const double* xr = (k & 1) ? p.xb : p.xa;
  if (s_status != kStatusTimeout)
    for (int64_t s = gw; s < p.nslices; s += nw) {
      const int64_t i = s * kSliceRows + lane;
      if (i < p.n) p.x_out[i] = xr[i];
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    jacobi_stats st;
    st.sweeps = k;
    st.outer_steps = 0;
    st.final_delta = s_delta;
    st.rel_residual = __longlong_as_double(0x7FF8000000000000ll);
    st.status = s_status;
    st.converged = s_status == kStatusOk;
    p.ctl->result = st;
    if (p.stats_out) *p.stats_out = st;
  }
}

// ------------------------------------------------------------------ mixed-precision refinement

template <class TV>
__device__ __forceinline__ float to_f32(TV v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <class TV>
__global__ void csr_narrow_kernel(const double* __restrict__ sval, int64_t slots, TV* tlo) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < slots;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float f = __double2float_rn(sval[e]);
    if constexpr (sizeof(TV) == 4)
      tlo[e] = f;
    else
      tlo[e] = __float2bfloat16_rn(f);
  }
}

// Grid-wide maxima of two per-thread values (IEEE bits of non-negative numbers) through rotating slot
// phase % 3 and one grid barrier; every thread returns with both maxima.  False on a timeout or another
// CTA's error.  Phase `phase` is recorded in the device trace with `kind`.
__device__ bool grid_max2(const CsrParams& p, uint32_t phase, int kind, unsigned long long& m0,
                          unsigned long long& m1, unsigned long long* s0, unsigned long long* s1, int* s_ok) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  m0 = warp_max_u64(m0);
  m1 = warp_max_u64(m1);
  if (lane == 0) {
    s0[warp] = m0;
    s1[warp] = m1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b0 = 0, b1 = 0;
    for (int q = 0; q < kCsrWarps; ++q) {
      b0 = s0[q] > b0 ? s0[q] : b0;
      b1 = s1[q] > b1 ? s1[q] : b1;
    }
    const int slot = static_cast<int>(phase % 3);
    if (b0) atomicMax(&p.ctl->red[slot][0], b0);
    if (b1) atomicMax(&p.ctl->red[slot][1], b1);
    if (blockIdx.x == 0) {
      p.ctl->red[(phase + 1) % 3][0] = 0ull;
      p.ctl->red[(phase + 1) % 3][1] = 0ull;
    }
    bool ok;
    if (p.test_skip_arrival && blockIdx.x == 0 && phase == 0) {
      ok = false;
      atomicMin(&p.ctl->status, kStatusTimeout);
    } else {
      ok = grid_arrive_and_wait(&p.ctl->arrive, &p.ctl->status, (phase + 1) * gridDim.x, p.wait_ns);
      if (!ok) atomicMin(&p.ctl->status, kStatusTimeout);
    }
    if (blockIdx.x == 0 && phase < static_cast<uint32_t>(kTraceCap)) {
      p.ctl->t_end[phase] = global_timer_ns();
      p.ctl->kind[phase] = kind;
      p.ctl->nphase = static_cast<int>(phase) + 1;
    }
    s0[0] = __ldcg(&p.ctl->red[slot][0]);
    s1[0] = __ldcg(&p.ctl->red[slot][1]);
    *s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  m0 = s0[0];
  m1 = s1[0];
  const bool ok = *s_ok != 0;
  __syncthreads();  // s0 / s1 are written again by the next call
  return ok;
}

// The refinement in one persistent launch.  Outer step: r' = c + T x' - x' with x' = x + delta (the last
// inner correction, gathered as x_j + delta_j, so no separate update pass), written as the FP32 right-hand
// side of the inner solve, with max |a_ii r'| / ||b||_inf as the stopping quantity (<= tol).  Inner sweeps:
// delta^(1) = r', delta^(l+1) = r' + T_lo delta^(l) in FP32, until the change is at most inner_rtol times the
// magnitude or max_inner sweeps.  Each phase ends with one grid barrier; every CTA takes the same decisions.
template <class TV, class F>
__global__ void __launch_bounds__(kCsrThreads, kCsrMinBlocks) csr_ir_kernel(CsrIrParams q) {
  const CsrParams& p = q.base;
  __shared__ unsigned long long s0[kCsrWarps], s1[kCsrWarps];
  __shared__ int s_ok;
  __shared__ int sdoff[kMaxDiag];
  load_doff(p, sdoff);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * kCsrWarps + warp;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kCsrWarps;
  const TV* tlo = static_cast<const TV*>(q.tlo);
  if (blockIdx.x == 0 && threadIdx.x == 0) p.ctl->t_start = global_timer_ns();

  uint32_t phase = 0;
  int outer = 0;
  int64_t inner_total = 0;
  double rel = 0.0;
  int status = kStatusNotConverged;
  const float* dcur = nullptr;  // correction not yet added to x
  const double* xc = p.xa;      // x
  double* xn = p.xb;            // x + delta
  for (;;) {
    // ---- FP64 residual of x' = x + delta
    unsigned long long mr = 0, unused = 0;
    for (int64_t s = gw; s < p.nslices; s += nw) {
      int64_t o0;
      const int w = F::width(p, s, o0);
      const int64_t i = s * kSliceRows + lane;
      const bool live = i < p.n;
      double xi = 0.0, acc = 0.0;
      if (live) {
        xi = __ldcg(xc + i) + (dcur ? static_cast<double>(__ldcg(dcur + i)) : 0.0);
        acc = __ldcs(p.c + i);
      }
#pragma unroll 4
      for (int t = 0; t < w; ++t) {
        const int64_t j = F::col(p, o0, t, lane, i, sdoff);
        const double xj = __ldcg(xc + j) + (dcur ? static_cast<double>(__ldcg(dcur + j)) : 0.0);
        acc = fma(__ldcs(p.sval + F::at(p, o0, t, lane)), xj, acc);
      }
      if (live) {
        const double r = acc - xi;
        xn[i] = xi;
        q.rf[i] = __double2float_rn(r);
        const unsigned long long b = abs_bits(__ldg(p.d + i) * r);
        mr = b > mr ? b : mr;
      }
    }
    const bool ok = grid_max2(p, phase++, JACOBI_PHASE_RESID64, mr, unused, s0, s1, &s_ok);
    rel = bits_to_double(mr) / p.bnorm;
    if (!ok) {
      status = kStatusTimeout;
      break;
    }
    if (!isfinite(rel)) {
      status = kStatusNonfinite;
      break;
    }
    if (rel <= p.tol) {
      status = kStatusOk;
      break;
    }
    if (outer >= q.max_outer) break;  // NOT_CONVERGED with x'
    ++outer;
    xc = xn;
    xn = xn == p.xa ? p.xb : p.xa;
    // ---- inner sweeps on the correction, FP32
    const float* dold = q.rf;
    float* dnew = q.da;
    bool timed_out = false;
    for (int l = 1;; ++l) {
      // maxima on FP32 bits (non-negative floats order like their bits, NaN above infinity), widened once
      // per thread: a widening per row would put two conversions per row on the FP64 pipe
      unsigned int fc = 0, fg = 0;
      int64_t s_first = gw;
      if constexpr (std::is_same<F, DiaFmt>::value) {
        // DIA: two slices per step (every slice has the same diagonals), their loads in flight together
        const int w = p.ndiag;
        for (; s_first + nw < p.nslices; s_first += 2 * nw) {
          const int64_t sa = s_first, sb = s_first + nw;
          const int64_t ia = sa * kSliceRows + lane, ib = sb * kSliceRows + lane;
          const bool la = ia < p.n, lb = ib < p.n;
          float acca = la ? __ldcg(q.rf + ia) : 0.0f, accb = lb ? __ldcg(q.rf + ib) : 0.0f;
          const TV* ta = tlo + sa * w * kSliceRows + lane;
          const TV* tb = tlo + sb * w * kSliceRows + lane;
#pragma unroll 4
          for (int t = 0; t < w; ++t) {
            const float va = to_f32<TV>(__ldcs(ta + kSliceRows * t)), vb = to_f32<TV>(__ldcs(tb + kSliceRows * t));
            const float ga = __ldcg(dold + ia + sdoff[t]), gb = __ldcg(dold + ib + sdoff[t]);
            acca = fmaf(va, ga, acca);
            accb = fmaf(vb, gb, accb);
          }
          if (la) {
            const float old = __ldcg(dold + ia);
            dnew[ia] = acca;
            const unsigned int b1 = __float_as_uint(fabsf(acca - old)), b2 = __float_as_uint(fabsf(acca));
            fc = b1 > fc ? b1 : fc;
            fg = b2 > fg ? b2 : fg;
          }
          if (lb) {
            const float old = __ldcg(dold + ib);
            dnew[ib] = accb;
            const unsigned int b1 = __float_as_uint(fabsf(accb - old)), b2 = __float_as_uint(fabsf(accb));
            fc = b1 > fc ? b1 : fc;
            fg = b2 > fg ? b2 : fg;
          }
        }
      }
      for (int64_t s = s_first; s < p.nslices; s += nw) {
        int64_t o0;
        const int w = F::width(p, s, o0);
        const int64_t i = s * kSliceRows + lane;
        const bool live = i < p.n;
        float acc = live ? __ldcg(q.rf + i) : 0.0f;
#pragma unroll 4
        for (int t = 0; t < w; ++t)
          acc = fmaf(to_f32<TV>(__ldcs(tlo + F::at(p, o0, t, lane))), __ldcg(dold + F::col(p, o0, t, lane, i, sdoff)),
                     acc);
        if (live) {
          const float old = __ldcg(dold + i);
          dnew[i] = acc;
          const unsigned int b1 = __float_as_uint(fabsf(acc - old)), b2 = __float_as_uint(fabsf(acc));
          fc = b1 > fc ? b1 : fc;
          fg = b2 > fg ? b2 : fg;
        }
      }
      unsigned long long mc = abs_bits(__uint_as_float(fc)), mg = abs_bits(__uint_as_float(fg));
      const bool iok = grid_max2(p, phase++, JACOBI_PHASE_INNER, mc, mg, s0, s1, &s_ok);
      ++inner_total;
      if (!iok) {
        timed_out = true;
        break;
      }
      const double ch = bits_to_double(mc), mag = bits_to_double(mg);
      if (!(ch > static_cast<double>(q.inner_rtol) * mag) || l >= q.max_inner) {  // NaN stops too
        dcur = dnew;
        break;
      }
      dold = dnew;
      dnew = dnew == q.da ? q.db : q.da;
    }
    if (timed_out) {
      status = kStatusTimeout;
      break;
    }
  }
  // x' of the last residual: converged, capped or non-finite alike
  if (status != kStatusTimeout)
    for (int64_t s = gw; s < p.nslices; s += nw) {
      const int64_t i = s * kSliceRows + lane;
      if (i < p.n) p.x_out[i] = xn[i];
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    jacobi_stats st;
    st.sweeps = inner_total;
    st.outer_steps = outer + 1;
    st.final_delta = rel;
    st.rel_residual = rel;
    st.status = status;
    st.converged = status == kStatusOk;
    p.ctl->result = st;
    if (p.stats_out) *p.stats_out = st;
  }
}

int blocks_for(int64_t items, int threads) { return static_cast<int>((items + threads - 1) / threads); }

}  // namespace

cudaError_t launch_csr_check(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                             const double* val, double* d, int32_t* lens, unsigned long long* key, cudaStream_t s) {
  csr_check_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, nnz, row_ptr, col_idx, val, d, lens, key);
  return cudaGetLastError();
}

cudaError_t launch_csr_widths(int64_t n, const int32_t* lens, int32_t* width, cudaStream_t s) {
  const int64_t nslices = (n + kSliceRows - 1) / kSliceRows;
  csr_widths_kernel<<<blocks_for(nslices * 32, 256), 256, 0, s>>>(n, nslices, lens, width);
  return cudaGetLastError();
}

cudaError_t launch_csr_fill(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                            const double* d, const int64_t* soff, double* sval, int32_t* scol, double* c,
                            unsigned long long* bmax, cudaStream_t s) {
  const int64_t nslices = (n + kSliceRows - 1) / kSliceRows;
  csr_fill_kernel<<<blocks_for(nslices * kSliceRows, 256), 256, 0, s>>>(n, nslices, row_ptr, col_idx, val, d, soff,
                                                                         sval, scol, c, bmax);
  return cudaGetLastError();
}

cudaError_t launch_csr_dia_check(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const int32_t* doff,
                                 int ndiag, int* bad, cudaStream_t s) {
  csr_dia_check_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, row_ptr, col_idx, doff, ndiag, bad);
  return cudaGetLastError();
}

cudaError_t launch_csr_dia_fill(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                                const double* d, const int32_t* doff, int ndiag, double* dval, double* c,
                                unsigned long long* bmax, cudaStream_t s) {
  csr_dia_fill_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, row_ptr, col_idx, val, d, doff, ndiag, dval, c, bmax);
  return cudaGetLastError();
}

namespace {
const void* solve_fn(bool resid, bool dia) {
  if (dia)
    return resid ? reinterpret_cast<const void*>(csr_solve_kernel<true, DiaFmt>)
                 : reinterpret_cast<const void*>(csr_solve_kernel<false, DiaFmt>);
  return resid ? reinterpret_cast<const void*>(csr_solve_kernel<true, EllFmt>)
               : reinterpret_cast<const void*>(csr_solve_kernel<false, EllFmt>);
}
const void* ir_fn(CsrInner kind, bool dia) {
  if (dia)
    return kind == CsrInner::F32 ? reinterpret_cast<const void*>(csr_ir_kernel<float, DiaFmt>)
                                 : reinterpret_cast<const void*>(csr_ir_kernel<__nv_bfloat16, DiaFmt>);
  return kind == CsrInner::F32 ? reinterpret_cast<const void*>(csr_ir_kernel<float, EllFmt>)
                               : reinterpret_cast<const void*>(csr_ir_kernel<__nv_bfloat16, EllFmt>);
}
// Co-resident grid of the kernels in fns (the smallest of their occupancies), capped at kMaxGrid.
int max_grid_of(std::initializer_list<const void*> fns) {
  int dev = 0, sms = 0, best = 1 << 30;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  for (const void* fn : fns) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCsrThreads, 0) != cudaSuccess) return 0;
    best = per_sm < best ? per_sm : best;
  }
  const int g = best * sms;
  return g < kMaxGrid ? g : kMaxGrid;
}
}  // namespace

cudaError_t launch_csr_solve(const CsrParams& p, int grid, cudaStream_t s) {
  CsrParams copy = p;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(solve_fn(p.norm == JACOBI_NORM_RESID, p.ndiag > 0), dim3(grid),
                                     dim3(kCsrThreads), args, 0, s);
}

int csr_max_grid() {
  // the instantiations may differ in registers: the smallest co-resident grid serves all of them
  return max_grid_of({solve_fn(false, false), solve_fn(true, false), solve_fn(false, true), solve_fn(true, true)});
}

int csr_warps_per_cta() { return kCsrWarps; }

cudaError_t launch_csr_narrow(CsrInner kind, const double* sval, int64_t slots, void* tlo, cudaStream_t s) {
  const int blocks = static_cast<int>(std::min<int64_t>((slots + 255) / 256, 65536));
  if (slots <= 0) return cudaSuccess;
  if (kind == CsrInner::F32)
    csr_narrow_kernel<float><<<blocks, 256, 0, s>>>(sval, slots, static_cast<float*>(tlo));
  else
    csr_narrow_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(sval, slots, static_cast<__nv_bfloat16*>(tlo));
  return cudaGetLastError();
}

cudaError_t launch_csr_ir_solve(CsrInner kind, const CsrIrParams& p, int grid, cudaStream_t s) {
  CsrIrParams copy = p;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(ir_fn(kind, p.base.ndiag > 0), dim3(grid), dim3(kCsrThreads), args, 0, s);
}

int csr_ir_max_grid(CsrInner kind) { return max_grid_of({ir_fn(kind, false), ir_fn(kind, true)}); }

}  // namespace jac
