// Gauss-Seidel / SOR sweeps for one dense system, the relaxed relative of the Section 2 iteration:
//
//   x_i^(k) = x_i^(k-1) + omega ( (beta_i - sum_{j<i} alpha_ij x_j^(k) - sum_{j>i} alpha_ij x_j^(k-1))
//                                 / alpha_ii - x_i^(k-1) ).
//
// The sweep is sequential in i, so it is distributed as a chain over row blocks: CTA c owns rows
// [r_c, r_(c+1)) and, in sweep k,
//   1. subtracts from u_i = beta_i the columns after its block (previous iterate) and the strict upper
//      part of its diagonal block (previous iterate) -- work that needs nobody else;
//   2. subtracts the columns of every earlier block as soon as that block publishes its new values (a
//      per-CTA flag set with release semantics after the block's x^(k) is in memory; read with acquire);
//      the previous block's columns, the last to arrive, come from a tile of A kept in shared memory;
//   3. solves its block: with M = D + omega L (the block's diagonal and strict lower part),
//      M x = (1 - omega) D x^(k-1) + omega u, i.e. x = M^-1 w with M^-1 formed once per solve in shared
//      memory;
//   4. writes x^(k) for its rows and publishes its flag.
// So the chain's critical path per block is two shared-memory matrix-vector products (the previous
// block's contribution and M^-1 w) and one flag hand-off; everything that streams A from HBM runs
// before the block's turn.
// The result is the sequential Gauss-Seidel / SOR sweep (up to rounding order), whatever the grid.
// Sweeps overlap: after publishing x^(k), a block starts sweep k+1's columns after it as the later blocks
// publish, and the stopping test on sweep k is read once the last block has published (no grid barrier).
// Every wait is bounded by %globaltimer; a wait that runs out sets JACOBI_ERR_TIMEOUT for the solve.
#include "device_util.cuh"
#include "gs.cuh"

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

// u[i] -= sum_{j in [c0, c1)} a_(r0+i),j x_j for the block's rows: each warp takes 4 rows at a time,
// lanes take column pairs (16-byte loads: rows start 16-byte aligned), with a scalar head and tail for
// odd ends.  x is read through L2 (other CTAs write it during the launch).
__device__ void rows_dot(const GsParams& p, int64_t r0, int m, int64_t c0, int64_t c1, const double* x, double* u,
                         int warp, int lane) {
  if (c1 <= c0) return;
  const int64_t jp = c0 + (c0 & 1);             // first even column
  const int64_t je = jp + ((c1 - jp) & ~int64_t(1));  // end of the pairs
  for (int i0 = 4 * warp; i0 < m; i0 += 4 * kGsWarps) {
    const int nr = m - i0 < 4 ? m - i0 : 4;
    const double* rp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) rp[q] = p.A + (r0 + i0 + (q < nr ? q : nr - 1)) * p.lda;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (lane == 0) {
      if (c0 & 1) {
        const double xv = __ldcg(x + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(__ldg(rp[q] + c0), xv, acc[q]);
      }
      if (je < c1) {
        const double xv = __ldcg(x + je);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(__ldg(rp[q] + je), xv, acc[q]);
      }
    }
#pragma unroll 2
    for (int64_t j = jp + 2 * lane; j < je; j += 64) {
      const double2 xv = __ldcg(reinterpret_cast<const double2*>(x + j));
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(rp[q] + j));
        acc[q] = fma(a.y, xv.y, fma(a.x, xv.x, acc[q]));
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = warp_sum(acc[q]);
    if (lane == 0)
      for (int q = 0; q < nr; ++q) u[i0 + q] -= acc[q];
  }
}

// u -= the columns of blocks [b0, b1) with x, taking each block once its flag reaches kf (in block order,
// runs of already-published blocks at once), and pulling the next awaited block into L2 meanwhile.
// Called by the whole CTA.  A wait that runs out clears *s_ok and skips the rest.
__device__ void process_published(const GsParams& p, int64_t r0, int m, int b0, int b1, int kf, const double* x,
                                  double* u, int warp, int lane, int* s_e, int* s_ok) {
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
    if (*s_ok) rows_dot(p, r0, m, p.n * done / G, p.n * e / G, x, u, warp, lane);
    done = e;
  }
}

__device__ __forceinline__ double bits_to_double(unsigned long long v) {
  return __longlong_as_double(static_cast<long long>(v));
}

__global__ void __launch_bounds__(kGsThreads) gs_solve_kernel(GsParams p) {
  extern __shared__ double sm[];
  constexpr int P = kGsPitch;
  double* dm = sm;                    // lower with diagonal: (M^-1)_ij; strict upper: a_(r0+i),(r0+j)
  double* pv = dm + kGsMaxRows * P;   // a_(r0+i),(s+j): this block's rows x the previous block's columns
  double* xo_b = pv + kGsMaxRows * P; // x^(k-1) of the block
  double* u = xo_b + kGsMaxRows;      // running right-hand side of the block's rows
  double* w = u + kGsMaxRows;         // M x = w
  double* xn_b = w + kGsMaxRows;      // x^(k) of the block
  double* xp = xn_b + kGsMaxRows;     // x^(k) of the previous block
  __shared__ unsigned long long s_red[kGsWarps];
  __shared__ double s_sq[kGsWarps];
  __shared__ int s_e, s_ok, s_next, s_status;

  const int G = gridDim.x, c = blockIdx.x;
  const int64_t r0 = p.n * c / G, r1 = p.n * (c + 1) / G;
  const int64_t sp = c > 0 ? p.n * (c - 1) / G : 0;  // first column of the previous block
  const int m = static_cast<int>(r1 - r0), mp = static_cast<int>(r0 - sp);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double om = p.omega;
  if (tid == 0 && c == 0) p.ctl->t_start = global_timer_ns();

  // ---- once per solve: M^-1 for M = D + omega L of the diagonal block (from the block staged in pv),
  // the block's strict upper part, then the previous block's columns
  for (int e = tid; e < m * m; e += kGsThreads) {
    const int i = e / m, j = e % m;
    pv[i * P + j] = p.A[(r0 + i) * p.lda + r0 + j];
  }
  __syncthreads();
  if (tid < m) {
    // column t by forward substitution: z_t = 1 / a_tt, z_i = -(sum_{t<=j<i} omega a_ij z_j) / a_ii
    const int t = tid;
    dm[t * P + t] = __ldg(p.rinv + r0 + t);
    for (int i = t + 1; i < m; ++i) {
      double s = 0.0;
      for (int j = t; j < i; ++j) s = fma(pv[i * P + j], dm[j * P + t], s);
      dm[i * P + t] = -(om * s) * __ldg(p.rinv + r0 + i);
    }
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += kGsThreads) {
    const int i = e / m, j = e % m;
    if (j > i) dm[i * P + j] = pv[i * P + j];
  }
  __syncthreads();
  for (int e = tid; e < m * mp; e += kGsThreads) {
    const int i = e / mp, j = e % mp;
    pv[i * P + j] = p.A[(r0 + i) * p.lda + sp + j];
  }
  __syncthreads();

  // ---- sweeps.  Iteration k ends with this block's x^(k) published, then already computes the part of
  // sweep k+1 that needs the previous iterate (the columns after the block, from x^(k) of the later
  // blocks, taken as they publish), and decides on sweep k once the last block has published it: every
  // block's change norm is in red[k % 3] / part by then (each block adds its own before publishing, and
  // the flags are released and acquired in chain order), so every CTA takes the same decision with no
  // grid barrier, and the next sweep's chain starts as soon as the last block of this one is done.
  // x^(k) lives in xb for odd k, xa for even k; x^(0) (the start vector) in xa
  int64_t k = 1;
  double delta = 0.0;
  int status = kStatusNotConverged;
  if (tid == 0) s_ok = 1;
  for (int i = tid; i < m; i += kGsThreads) {
    xo_b[i] = __ldcg(p.xa + r0 + i);
    u[i] = __ldg(p.b + r0 + i);
  }
  __syncthreads();
  rows_dot(p, r0, m, r1, p.n, p.xa, u, warp, lane);  // sweep 1: the later blocks' x^(0) is the input
  for (;; ++k) {
    double* xn = (k & 1) ? p.xb : p.xa;
    __syncthreads();
    // the block's strict upper part, with x^(k-1)
    for (int i = warp; i < m; i += kGsWarps) {
      double s = 0.0;
      for (int j = i + 1 + lane; j < m; j += 32) s = fma(dm[i * P + j], xo_b[j], s);
      s = warp_sum(s);
      if (lane == 0) u[i] -= s;
    }
    // the blocks before the previous one, with x^(k), as they are published (in order)
    process_published(p, r0, m, 0, c - 1, static_cast<int>(k), xn, u, warp, lane, &s_e, &s_ok);
    //    and the previous block's columns from the shared-memory tile
    if (c > 0) {
      __syncthreads();
      if (tid == 0 && s_ok && !wait_flag(p.flags + c - 1, static_cast<int>(k), &p.ctl->status, p.wait_ns)) s_ok = 0;
      __syncthreads();
      for (int j = tid; j < mp; j += kGsThreads) xp[j] = __ldcg(xn + sp + j);
      __syncthreads();
      for (int i2 = tid; i2 < 2 * kGsMaxRows; i2 += kGsThreads) {  // two threads per row, even / odd columns
        const int i = i2 >> 1;
        double s = 0.0;
        if (i < m)
          for (int j = i2 & 1; j < mp; j += 2) s = fma(pv[i * P + j], xp[j], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (i < m && (i2 & 1) == 0) u[i] -= s;
      }
    }
    __syncthreads();
    // x^(k) = M^-1 w, w = (1 - omega) D x^(k-1) + omega u
    for (int i = tid; i < m; i += kGsThreads)
      w[i] = om == 1.0 ? u[i] : fma(1.0 - om, __ldg(p.d + r0 + i) * xo_b[i], om * u[i]);
    __syncthreads();
    unsigned long long mx = 0;
    double sq = 0.0;
    for (int i2 = tid; i2 < 2 * kGsMaxRows; i2 += kGsThreads) {  // two threads per row
      const int i = i2 >> 1;
      double x = 0.0;
      if (i < m)
        for (int j = i2 & 1; j <= i; j += 2) x = fma(dm[i * P + j], w[j], x);
      x += __shfl_xor_sync(0xffffffffu, x, 1);
      if (i < m && (i2 & 1) == 0) {
        xn_b[i] = x;
        xn[r0 + i] = x;
        const double diff = x - xo_b[i];
        const unsigned long long bb = abs_bits(diff);
        mx = bb > mx ? bb : mx;
        sq = fma(diff, diff, sq);
      }
    }
    // the block's change norm, then x^(k) published
    mx = warp_max_u64(mx);
    sq = warp_sum(sq);
    if (lane == 0) {
      s_red[warp] = mx;
      s_sq[warp] = sq;
    }
    __syncthreads();
    const int slot = static_cast<int>(k % 3);
    if (tid == 0) {
      unsigned long long bm = 0;
      double bs = 0.0;
      for (int q = 0; q < kGsWarps; ++q) {  // fixed order
        bm = s_red[q] > bm ? s_red[q] : bm;
        bs += s_sq[q];
      }
      if (c == 0) p.ctl->red[slot][0] = 0ull;  // the first block of the sweep opens its slot
      if (p.norm == JACOBI_NORM_2)
        p.part[slot * kMaxGrid + c] = bs;
      else if (bm)
        atomicMax(&p.ctl->red[slot][0], bm);
      if (!s_ok) atomicMin(&p.ctl->status, kStatusTimeout);
      __threadfence();
      st_release_i32(p.flags + c, static_cast<int>(k));
    }
    // sweep k+1's columns after the block, from x^(k) of the later blocks as they publish
    for (int i = tid; i < m; i += kGsThreads) {
      xo_b[i] = xn_b[i];
      u[i] = __ldg(p.b + r0 + i);
    }
    process_published(p, r0, m, c + 1, G, static_cast<int>(k), xn, u, warp, lane, &s_e, &s_ok);
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
