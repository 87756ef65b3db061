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
                                int32_t* scol, double* c) {
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
    c[i] = c[i] / di;  // c_i = b_i / a_ii (c holds b on entry)
  }
  const int32_t self = static_cast<int32_t>(i < n ? i : n - 1);
  for (; t < w; ++t) {
    sval[base + kSliceRows * t] = 0.0;
    scol[base + kSliceRows * t] = self;
  }
}

__device__ __forceinline__ double bits_to_double(unsigned long long v) {
  return __longlong_as_double(static_cast<long long>(v));
}

__global__ void __launch_bounds__(kCsrThreads, kCsrMinBlocks) csr_solve_kernel(CsrParams p) {
  __shared__ unsigned long long s_mx[kCsrWarps];
  __shared__ double s_sq[kCsrWarps];
  __shared__ int s_next, s_status;
  __shared__ double s_delta;
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
      const int64_t o0 = __ldg(p.soff + s), o1 = __ldg(p.soff + s + 1);
      const int w = static_cast<int>((o1 - o0) / kSliceRows);
      // pull the warp's next slice into L2 meanwhile: its values and columns, one 128-byte line per lane
      if (s + nw < p.nslices) {
        const int64_t q0 = __ldg(p.soff + s + nw), q1 = __ldg(p.soff + s + nw + 1);
        const int64_t vl = (q1 - q0) / 16, cl = (q1 - q0) / 32;  // lines of values (8 B) and columns (4 B)
        for (int64_t l = lane; l < vl + cl; l += 32) {
          const char* a = l < vl ? reinterpret_cast<const char*>(p.sval + q0) + 128 * l
                                 : reinterpret_cast<const char*>(p.scol + q0) + 128 * (l - vl);
          asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
        }
      }
      const int64_t i = s * kSliceRows + lane;
      const bool live = i < p.n;
      const double xo = live ? __ldcg(xc + i) : 0.0;
      const double* v = p.sval + o0 + lane;
      const int32_t* cc = p.scol + o0 + lane;
      double x = live ? __ldcs(p.c + i) : 0.0;
#pragma unroll 4
      for (int t = 0; t < w; ++t) x = fma(__ldcs(v + kSliceRows * t), __ldcg(xc + __ldcs(cc + kSliceRows * t)), x);
      if (live) {
        const double diff = x - xo;
        xn[i] = x;
        const unsigned long long bb = abs_bits(diff);
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
                            cudaStream_t s) {
  const int64_t nslices = (n + kSliceRows - 1) / kSliceRows;
  csr_fill_kernel<<<blocks_for(nslices * kSliceRows, 256), 256, 0, s>>>(n, nslices, row_ptr, col_idx, val, d, soff,
                                                                         sval, scol, c);
  return cudaGetLastError();
}

cudaError_t launch_csr_solve(const CsrParams& p, int grid, cudaStream_t s) {
  CsrParams copy = p;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(csr_solve_kernel), dim3(grid), dim3(kCsrThreads),
                                     args, 0, s);
}

int csr_max_grid() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_solve_kernel, kCsrThreads, 0) != cudaSuccess)
    return 0;
  const int g = per_sm * sms;
  return g < kMaxGrid ? g : kMaxGrid;
}

int csr_warps_per_cta() { return kCsrWarps; }

}  // namespace jac
