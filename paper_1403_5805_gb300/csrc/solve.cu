// Persistent Jacobi solve kernels for GB300 (sm_103a).
//
// One cooperative launch runs a whole solve.  Each CTA owns a contiguous block of rows (the paper's
// row-wise distribution of Section 3.1, here over the SMs of one GPU).  Per sweep it streams its rows
// of the matrix from HBM exactly once through a shared-memory ring: one producer warp issues 1-D TMA
// bulk copies (one row segment of a column chunk each, 16 rows per ring item, 3 items of 56 KB) that
// complete on mbarriers; fourteen consumer warps (7 column slices x 2 groups of 8 rows) read them with
// 128-bit shared-memory loads and accumulate row dot products against the current iterate (read from
// L2), reduce them with warp shuffles and a fixed-order cross-warp sum, and apply the component update
// of Section 2 in the epilogue.  When a CTA's rows fit in the ring (small systems), later sweeps reuse
// them from shared memory.  A handle's first BF16 / FP32 inner sweep streams FP64 A instead and writes
// the narrow copy as it sweeps.  The max-norm change is reduced in the
// same epilogue (order-free integer max on the IEEE bits), combined over the grid with one atomic and
// one grid barrier per sweep, and every CTA takes the same stop decision from it - the stopping test
// of the Section 2 algorithm with no host round trip.
//
// Kernels
//   fp64_solve_kernel        X^(k) = D^-1 (B - (A - D) X^(k-1)), all FP64 (Section 2 update).
//   ir_solve_kernel<Narrow>  FP64 iterative refinement around inner Jacobi sweeps on a narrow copy of
//                            the off-diagonal part of A (FP32 / BF16 / E4M3 + row scale), FP32
//                            accumulation; FP64 residual r = B - A X and update X += delta.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "device_util.cuh"
#include "dot.cuh"
#include "solver.cuh"
#include "splitfloat.cuh"

#include <type_traits>

namespace jac {
namespace {

struct Ring {
  uint64_t full[kStages];   // producer -> consumers: stage filled (1 arrival + transaction bytes)
  uint64_t empty[kStages];  // consumers -> producer: stage free again (one arrival per consumer warp)
};

template <typename TM>
__host__ __device__ constexpr int chunk_cols() {
  return kColWarps * 32 * MatTraits<TM>::kVec;
}

struct Block {
  Ring* ring;
  char* stages;
  volatile int* abort;   // CTA-wide abort flag (shared memory)
  int* gstatus;          // grid-wide status word (Ctl::status)
  uint64_t wait_ns;      // limit of every wait
  int drop_first;        // test only: announce ring item 0 without copying it
};

__device__ __forceinline__ void raise_abort(const Block& B) {
  *B.abort = 1;
  atomicCAS(B.gstatus, 0, kStatusTimeout);
}

// Producer warp: stream rows [r0, r1) of M (columns [0, n)) into the ring, one item per (row group,
// column chunk).  u counts ring items over the whole kernel (shared by producer and consumers).
template <typename TM>
__device__ void produce_phase(const Block& B, uint32_t& u, const TM* M, int64_t ld, int64_t n,
                              int64_t r0, int64_t r1) {
  constexpr int K = chunk_cols<TM>();
  const int lane = threadIdx.x & 31;
  const int64_t nch = (n + K - 1) / K;
  // order this phase's bulk copies after generic-proxy writes of the matrix seen at the last grid barrier
  // (the narrow copy written by a fused first inner sweep)
  fence_proxy_async_global();
  for (int64_t g0 = r0; g0 < r1; g0 += kRows) {
    const int rows = static_cast<int>(i64min(kRows, r1 - g0));
    for (int64_t c = 0; c < nch; ++c) {
      const int s = static_cast<int>(u % kStages);
      const uint32_t par = ((u / kStages) & 1u) ^ 1u;
      const int64_t j0 = c * K;
      const int64_t wcols = i64min(K, n - j0);
      const uint32_t rbytes = static_cast<uint32_t>((wcols * static_cast<int64_t>(sizeof(TM)) + 15) & ~int64_t(15));
      int ok = 1;
      if (lane == 0) {
        // abort is re-read after the wait: consumers that gave up raise it before they release the stage,
        // and a stage whose previous item never arrived must not be armed again
        ok = (*B.abort == 0) && mbar_wait(&B.ring->empty[s], par, B.wait_ns) && (*B.abort == 0);
        if (ok) mbar_arrive_expect_tx(&B.ring->full[s], rbytes * static_cast<uint32_t>(rows));
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) raise_abort(B);
        return;
      }
      if (lane < rows && !(B.drop_first && u == 0))
        bulk_copy_g2s(B.stages + s * kStageBytes + lane * kRowBytes, M + (g0 + lane) * ld + j0, rbytes,
                      &B.ring->full[s]);
      ++u;
    }
  }
}

// Sum each of the 8 per-lane accumulators over the 32 lanes of a warp in 9 shuffle+add steps: every
// exchange halves the values a lane keeps, so after the xor-16/8/4 steps lane l holds the partial of row
// row_of_lane(l) over 8 lanes, and the xor-2/1 steps finish it.  The order of additions is fixed.
template <typename Acc>
__device__ __forceinline__ Acc transpose_reduce8(const Acc (&v)[kRowsPerWarp], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  Acc w4[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const Acc send = b4 ? v[r] : v[r + 4];
    const Acc keep = b4 ? v[r + 4] : v[r];
    w4[r] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  Acc w2[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const Acc send = b3 ? w4[r] : w4[r + 2];
    const Acc keep = b3 ? w4[r + 2] : w4[r];
    w2[r] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const Acc send = b2 ? w2[0] : w2[1];
  const Acc keep = b2 ? w2[1] : w2[0];
  Acc w1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  w1 += __shfl_xor_sync(0xffffffffu, w1, 2);
  w1 += __shfl_xor_sync(0xffffffffu, w1, 1);
  return w1;
}
__device__ __forceinline__ int row_of_lane(int lane) {
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// Consumer warps: row dot products of rows [r0, r1) against x, then epi.row(i, dot) by warp 0, lane
// (i - group start); epi.prefetch(i) runs on the same lane when the group starts, so the epilogue's
// operands arrive while the group streams.  Warp w covers column slice w % kColWarps of every chunk
// and rows [8 * (w / kColWarps), +8) of the group.  with_matrix == false skips the matrix (dot = 0).
// kResident: the ring items of this CTA's rows were loaded by an earlier phase and stay in their stages
// (every item of the phase has its own stage), so there is nothing to wait for and nothing to release.
template <typename TM, typename Epi, bool kResident = false>
__device__ void consume_phase(const Block& B, uint32_t& u, const typename MatTraits<TM>::X* x, int64_t n,
                              int64_t r0, int64_t r1, bool with_matrix,
                              typename MatTraits<TM>::Acc (*red)[kConsumerWarps][kRowsPerWarp], Epi& epi) {
  using XT = typename MatTraits<TM>::X;
  using Acc = typename MatTraits<TM>::Acc;
  constexpr int V = MatTraits<TM>::kVec;
  constexpr int K = chunk_cols<TM>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cw = warp % kColWarps, rh = warp / kColWarps;
  const int co = (cw * 32 + lane) * V;  // first column of this lane inside a chunk
  const int64_t nch = with_matrix ? (n + K - 1) / K : 0;
  int grp = 0;
  for (int64_t g0 = r0; g0 < r1; g0 += kRows, ++grp) {
    const int rows = static_cast<int>(i64min(kRows, r1 - g0));
    const int myrows = rows - rh * kRowsPerWarp;  // rows of this warp's half that exist (may be <= 0)
    if (warp == 0 && lane < rows) epi.prefetch(g0 + lane);
    Acc acc[kRowsPerWarp];
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r) acc[r] = Acc(0);
    XT xv[V], xn[V];
    if (nch > 0 && co < n) load_x(xv, x + co);
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t col = c * K + co;
      const int64_t ncol = col + K;
      if (c + 1 < nch && ncol < n) load_x(xn, x + ncol);  // prefetch the next chunk's x
      const int s = static_cast<int>(u % kStages);
      const uint32_t par = (u / kStages) & 1u;
      bool ok = (*B.abort == 0);
      if (ok && !kResident) ok = mbar_wait(&B.ring->full[s], par, B.wait_ns);
      if (!ok) {
        raise_abort(B);
      } else if (col < n && myrows > 0) {
        const char* base = B.stages + s * kStageBytes + rh * kRowsPerWarp * kRowBytes +
                           co * static_cast<int>(sizeof(TM));
        if (std::is_same<TM, double>::value && col + V <= n && myrows >= kRowsPerWarp) {
          // full rows of a full group: all loads first, then the rows' products interleaved, so a warp has
          // kRowsPerWarp independent accumulations in flight (each row's order of operations is unchanged)
          uint4 m[kRowsPerWarp];
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r) m[r] = *reinterpret_cast<const uint4*>(base + r * kRowBytes);
          seg_dot_rows(acc, m, xv);
        } else if (col + V <= n) {
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r)
            if (r < myrows) {
              const uint4 m = *reinterpret_cast<const uint4*>(base + r * kRowBytes);
              seg_dot(acc[r], m, xv);
            }
        } else {
          mask_tail(xv, col, n);
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r)
            if (r < myrows) {
              const uint4 m = *reinterpret_cast<const uint4*>(base + r * kRowBytes);
              seg_dot_tail(acc[r], m, xv, n - col);
            }
        }
      }
      __syncwarp();
      if (lane == 0 && !kResident) mbar_arrive(&B.ring->empty[s]);
      ++u;
#pragma unroll
      for (int e = 0; e < V; ++e) xv[e] = xn[e];
    }
    const Acc part = transpose_reduce8(acc, lane);
    if ((lane & 3) == 0) red[grp & 1][warp][row_of_lane(lane)] = part;
    // one barrier per group: red is double-buffered, and a buffer is rewritten only two groups later,
    // after every warp has passed the next group's barrier (so warp 0 has finished reading it)
    named_barrier(1, kConsumers);
    if (warp == 0 && lane < rows) {
      const int half = lane / kRowsPerWarp, r = lane % kRowsPerWarp;
      Acc dot = red[grp & 1][half * kColWarps][r];
#pragma unroll
      for (int w = 1; w < kColWarps; ++w) dot += red[grp & 1][half * kColWarps + w][r];  // fixed order
      epi.row(g0 + lane, dot);
    }
  }
}

// Same schedule as consume_phase<double> (ring items, warp layout, transposed reduction, epilogue),
// with the split-float arithmetic above.
template <typename Epi>
__device__ void consume_phase_split(const Block& B, uint32_t& u, const float2* xs, int g, int64_t n, int64_t r0,
                                    int64_t r1, const int* rexp, double (*red)[kConsumerWarps][kRowsPerWarp],
                                    Epi& epi) {
  constexpr int V = 2;
  constexpr int K = chunk_cols<double>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cw = warp % kColWarps, rh = warp / kColWarps;
  const int co = (cw * 32 + lane) * V;
  const int64_t nch = (n + K - 1) / K;
  int grp = 0;
  for (int64_t g0 = r0; g0 < r1; g0 += kRows, ++grp) {
    const int rows = static_cast<int>(i64min(kRows, r1 - g0));
    const int myrows = rows - rh * kRowsPerWarp;
    if (warp == 0 && lane < rows) epi.prefetch(g0 + lane);
    int sh[kRowsPerWarp];
    FF acc[kRowsPerWarp];
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r) {
      const int64_t row = g0 + rh * kRowsPerWarp + r;
      sh[r] = r < myrows ? __ldg(rexp + row) : 0;
      acc[r] = FF{0.0f, 0.0f};
    }
    // (hi, lo) of x_col and x_col+1; entries past n are zero (the split buffers' padding)
    float4 xv = make_float4(0.f, 0.f, 0.f, 0.f), xn = xv;
    if (nch > 0 && co < n) xv = __ldcg(reinterpret_cast<const float4*>(xs + co));
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t col = c * K + co;
      const int64_t ncol = col + K;
      if (c + 1 < nch && ncol < n) xn = __ldcg(reinterpret_cast<const float4*>(xs + ncol));
      const int s = static_cast<int>(u % kStages);
      const uint32_t par = (u / kStages) & 1u;
      bool ok = (*B.abort == 0);
      if (ok) ok = mbar_wait(&B.ring->full[s], par, B.wait_ns);
      if (!ok) {
        raise_abort(B);
      } else if (col < n && myrows > 0) {
        const bool two = col + 1 < n;  // the straddling segment's padding element is skipped
        const char* base = B.stages + s * kStageBytes + rh * kRowsPerWarp * kRowBytes + co * 8;
        if (two && myrows >= kRowsPerWarp) {
          // full group, both elements: the rows' steps interleaved (each row's order unchanged)
          uint4 m[kRowsPerWarp];
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r) m[r] = *reinterpret_cast<const uint4*>(base + r * kRowBytes);
          float ah[kRowsPerWarp], al[kRowsPerWarp];
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r)
            split_scaled(__hiloint2double(static_cast<int>(m[r].y), static_cast<int>(m[r].x)), sh[r], ah[r], al[r]);
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r) ff_fma(acc[r], ah[r], al[r], xv.x, xv.y);
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r)
            split_scaled(__hiloint2double(static_cast<int>(m[r].w), static_cast<int>(m[r].z)), sh[r], ah[r], al[r]);
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r) ff_fma(acc[r], ah[r], al[r], xv.z, xv.w);
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r) ff_renorm(acc[r]);
        } else {
#pragma unroll
          for (int r = 0; r < kRowsPerWarp; ++r)
            if (r < myrows) {
              const uint4 m = *reinterpret_cast<const uint4*>(base + r * kRowBytes);
              float ah, al;
              split_scaled(__hiloint2double(static_cast<int>(m.y), static_cast<int>(m.x)), sh[r], ah, al);
              ff_fma(acc[r], ah, al, xv.x, xv.y);
              if (two) {
                split_scaled(__hiloint2double(static_cast<int>(m.w), static_cast<int>(m.z)), sh[r], ah, al);
                ff_fma(acc[r], ah, al, xv.z, xv.w);
              }
              ff_renorm(acc[r]);
            }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.ring->empty[s]);
      ++u;
      xv = xn;
    }
    double dv[kRowsPerWarp];
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r)  // back to FP64, scaled by 2^(sh + g) (exact)
      dv[r] = (static_cast<double>(acc[r].hi) + static_cast<double>(acc[r].lo)) * pow2(sh[r]) * pow2(g);
    const double part = transpose_reduce8(dv, lane);
    if ((lane & 3) == 0) red[grp & 1][warp][row_of_lane(lane)] = part;
    named_barrier(1, kConsumers);
    if (warp == 0 && lane < rows) {
      const int half = lane / kRowsPerWarp, r = lane % kRowsPerWarp;
      double dot = red[grp & 1][half * kColWarps][r];
#pragma unroll
      for (int w = 1; w < kColWarps; ++w) dot += red[grp & 1][half * kColWarps + w][r];
      epi.row(g0 + lane, dot);
    }
  }
}

// The narrow copy of two FP64 entries of a row (FP64 -> FP32 -> TL, both to nearest even, the setup's
// rounding), stored at dst, and the two values as FP32.
__device__ __forceinline__ float2 store_narrow_pair(__nv_bfloat16* dst, float f0, float f1) {
  const __nv_bfloat162 q = __floats2bfloat162_rn(f0, f1);
  *reinterpret_cast<__nv_bfloat162*>(dst) = q;
  return __bfloat1622float2(q);
}
__device__ __forceinline__ float2 store_narrow_pair(float* dst, float f0, float f1) {
  *reinterpret_cast<float2*>(dst) = make_float2(f0, f1);
  return make_float2(f0, f1);
}

// First inner sweep of a solve on a handle whose narrow copy is not written yet: the ring streams FP64 A
// (items of consume_phase<double>), each lane rounds its two entries of every row to the narrow type,
// stores them (zero on the diagonal and in the row padding up to ldn), and accumulates the inner-sweep
// dot product of the rounded values with x in FP32.  The reduction and epilogue are consume_phase's.
template <typename TL, typename Epi>
__device__ void consume_phase_narrow(const Block& B, uint32_t& u, const float* x, int64_t n, int64_t r0, int64_t r1,
                                     TL* N, int64_t ldn, float (*red)[kConsumerWarps][kRowsPerWarp], Epi& epi) {
  constexpr int K = chunk_cols<double>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cw = warp % kColWarps, rh = warp / kColWarps;
  const int co = (cw * 32 + lane) * 2;  // first of this lane's two columns inside a chunk
  const int64_t nch = (n + K - 1) / K;  // K is a multiple of 16, so the chunks also cover the padding to ldn
  int grp = 0;
  for (int64_t g0 = r0; g0 < r1; g0 += kRows, ++grp) {
    const int rows = static_cast<int>(i64min(kRows, r1 - g0));
    const int myrows = rows - rh * kRowsPerWarp;
    if (warp == 0 && lane < rows) epi.prefetch(g0 + lane);
    const int64_t i0 = g0 + rh * kRowsPerWarp;  // this warp's first row
    float acc[kRowsPerWarp];
#pragma unroll
    for (int r = 0; r < kRowsPerWarp; ++r) acc[r] = 0.0f;
    // x[col], x[col + 1] (the iterate buffers are zero past n up to their padded length)
    float2 xv = make_float2(0.f, 0.f), xn = xv;
    if (nch > 0 && co < n) xv = __ldcg(reinterpret_cast<const float2*>(x + co));
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t col = c * K + co;
      const int64_t ncol = col + K;
      xn = make_float2(0.f, 0.f);
      if (c + 1 < nch && ncol < n) xn = __ldcg(reinterpret_cast<const float2*>(x + ncol));
      const int s = static_cast<int>(u % kStages);
      const uint32_t par = (u / kStages) & 1u;
      bool ok = (*B.abort == 0);
      if (ok) ok = mbar_wait(&B.ring->full[s], par, B.wait_ns);
      if (!ok) {
        raise_abort(B);
      } else if (col < ldn && myrows > 0) {
        const char* base = B.stages + s * kStageBytes + rh * kRowsPerWarp * kRowBytes + co * 8;
#pragma unroll
        for (int r = 0; r < kRowsPerWarp; ++r)
          if (r < myrows) {
            const int64_t i = i0 + r;
            float f0 = 0.0f, f1 = 0.0f;
            if (col < n) {  // entries at or past n were not copied into the stage (and may be anything in A)
              const uint4 m = *reinterpret_cast<const uint4*>(base + r * kRowBytes);
              if (col != i) f0 = __double2float_rn(__hiloint2double(static_cast<int>(m.y), static_cast<int>(m.x)));
              if (col + 1 < n && col + 1 != i)
                f1 = __double2float_rn(__hiloint2double(static_cast<int>(m.w), static_cast<int>(m.z)));
            }
            const float2 q = store_narrow_pair(N + i * ldn + col, f0, f1);
            if (col < n) {
              acc[r] = fmaf(q.x, xv.x, acc[r]);
              acc[r] = fmaf(q.y, xv.y, acc[r]);
            }
          }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.ring->empty[s]);
      ++u;
      xv = xn;
    }
    const float part = transpose_reduce8(acc, lane);
    if ((lane & 3) == 0) red[grp & 1][warp][row_of_lane(lane)] = part;
    named_barrier(1, kConsumers);
    if (warp == 0 && lane < rows) {
      const int half = lane / kRowsPerWarp, r = lane % kRowsPerWarp;
      float dot = red[grp & 1][half * kColWarps][r];
#pragma unroll
      for (int w = 1; w < kColWarps; ++w) dot += red[grp & 1][half * kColWarps + w][r];  // fixed order
      epi.row(g0 + lane, dot);
    }
  }
  // the narrow copy was written through the generic proxy and is read by bulk copies in later phases
  fence_proxy_async_global();
}

// Wait for every bulk copy this producer issued (the last kStages items) before the CTA exits.
__device__ void drain_ring(const Block& B, uint32_t u_issued) {
  const uint32_t first = u_issued > kStages ? u_issued - kStages : 0;
  for (uint32_t v = first; v < u_issued; ++v) mbar_wait(&B.ring->full[v % kStages], (v / kStages) & 1u, B.wait_ns);
}

__device__ __forceinline__ void init_ring(Ring* ring) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&ring->full[s], 1);
      mbar_init(&ring->empty[s], kConsumerWarps);
    }
    mbar_init_fence();
  }
}

__device__ __forceinline__ double bits_to_double(unsigned long long v) {
  return __longlong_as_double(static_cast<long long>(v));
}

__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) {
  return __ldcg(p);
}

// Publish this CTA's reduction values into slot (phase % 3), clear the slot of phase + 1, and wait at
// the grid barrier.  Called by lane 0 of warp 0.  Returns false on timeout / remote error.
__device__ bool publish_and_sync(Ctl* ctl, uint32_t phase, unsigned long long v0, unsigned long long v1,
                                 uint64_t wait_ns) {
  const int slot = static_cast<int>(phase % 3);
  if (v0) atomicMax(&ctl->red[slot][0], v0);
  if (v1) atomicMax(&ctl->red[slot][1], v1);
  if (blockIdx.x == 0) {
    const int nxt = static_cast<int>((phase + 1) % 3);
    ctl->red[nxt][0] = 0ull;
    ctl->red[nxt][1] = 0ull;
  }
  return grid_arrive_and_wait(&ctl->arrive, &ctl->status, (phase + 1) * gridDim.x, wait_ns);
}

// Device-side trace (CTA 0, lane 0 of warp 0): end time of phase `phase` and its kind.
__device__ __forceinline__ void trace_phase(Ctl* ctl, uint32_t phase, int kind) {
  if (blockIdx.x == 0 && phase < static_cast<uint32_t>(kTraceCap)) {
    ctl->t_end[phase] = global_timer_ns();
    ctl->kind[phase] = kind;
    ctl->nphase = static_cast<int>(phase) + 1;
  }
}

__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// ================================================================================ FP64 path

struct Fp64SweepEpi {
  const double* b;
  const double* d;
  const double* rinv;
  const double* xc;  // X^(k-1)
  double* xn;        // X^(k)
  int norm;
  unsigned long long mx;  // running max (bits) over this lane's rows
  double sq;              // running sum of squares (Euclidean norm)
  double pb, pd, pr, px;  // this lane's row operands, loaded when its row group starts
  __device__ __forceinline__ void prefetch(int64_t i) {
    pb = b[i];
    pd = d[i];
    pr = rinv[i];
    px = __ldcg(xc + i);
  }
  __device__ __forceinline__ void row(int64_t i, double dot) {
    const double s = fma(-pd, px, dot);  // sum_{j != i} a_ij x_j: the diagonal term taken back out
    const double xi = (pb - s) * pr;     // Section 2 component update, 1/a_ii precomputed
    xn[i] = xi;
    const double diff = xi - px;
    if (norm == JACOBI_NORM_RESID)
      mx = umax(mx, abs_bits(pd * diff));
    else
      mx = umax(mx, abs_bits(diff));
    sq = fma(diff, diff, sq);
  }
};

enum Next : int { kContinue = 0, kStop = 1 };

__global__ void __maxnreg__(kMaxRegs) fp64_solve_kernel(SolveParams p) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ Ring ring;
  __shared__ double red[2][kConsumerWarps][kRowsPerWarp];
  __shared__ int s_abort, s_next;
  char* stages = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));

  const int G = gridDim.x;
  const int64_t r0 = p.n * blockIdx.x / G, r1 = p.n * (blockIdx.x + 1) / G;
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_next = kContinue;
    if (blockIdx.x == 0) p.ctl->t_start = global_timer_ns();
  }
  init_ring(&ring);
  __syncthreads();
  Block B{&ring, stages, &s_abort, &p.ctl->status, p.wait_ns, p.test_drop_copy};
  const bool producer = threadIdx.x >= kConsumers;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  uint32_t u = 0;
  int cur = 0;                    // buffer holding X^(k-1): 0 -> xa, 1 -> xb
  int64_t k = 1;
  // Small systems: when every ring item of this CTA's rows has a stage of its own, the first sweep loads
  // them and later sweeps reuse them from shared memory (A does not change between sweeps), so a sweep
  // reads only the iterate from L2.
  const int64_t items = (r1 - r0 + kRows - 1) / kRows * ((p.n + chunk_cols<double>() - 1) / chunk_cols<double>());
  const bool resident = items <= kStages;
  double delta = 0.0;
  int status = kStatusNotConverged;
  for (;; ++k) {
    const double* xc = cur ? p.xb : p.xa;
    double* xn = cur ? p.xa : p.xb;
    Fp64SweepEpi epi{p.b, p.d, p.rinv, xc, xn, p.norm, 0ull, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (resident && k > 1) {
      if (!producer) {
        uint32_t u0 = 0;  // the stages of the first sweep's items, in the same order
        consume_phase<double, Fp64SweepEpi, true>(B, u0, xc, p.n, r0, r1, true, red, epi);
      }
    } else if (producer) {
      produce_phase<double>(B, u, p.A, p.lda, p.n, r0, r1);
    } else {
      consume_phase<double>(B, u, xc, p.n, r0, r1, true, red, epi);
    }
    __syncthreads();
    if (warp == 0) {
      // CTA reduction over warp 0 (lanes that own rows hold the running values)
      const unsigned long long mx = warp_max_u64(epi.mx);
      const double sq = warp_sum(epi.sq);
      const uint32_t phase = static_cast<uint32_t>(k - 1);
      int ok = 1;
      if (lane == 0) {
        if (p.norm == JACOBI_NORM_2) p.part[(k & 1) * kMaxGrid + blockIdx.x] = sq;
        ok = (s_abort == 0) && publish_and_sync(p.ctl, phase, p.norm == JACOBI_NORM_2 ? 0ull : mx, 0ull, p.wait_ns);
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();  // order the other lanes' reads after lane 0's acquire of the grid barrier
      double dk;
      if (p.norm == JACOBI_NORM_2) {
        double acc = 0.0;
        for (int j = lane; j < G; j += 32) acc += __ldcg(p.part + (k & 1) * kMaxGrid + j);
        dk = sqrt(warp_sum(acc));
      } else {
        dk = bits_to_double(ld_cg_u64(&p.ctl->red[phase % 3][0]));
        if (p.norm == JACOBI_NORM_RESID) dk = dk / __ldg(p.bnorm);
      }
      if (lane == 0) {
        trace_phase(p.ctl, phase, JACOBI_PHASE_SWEEP64);
        int next = kContinue;
        if (!ok) {
          status = kStatusTimeout;
          next = kStop;
        } else if (!isfinite(dk)) {
          status = kStatusNonfinite;
          next = kStop;
        } else if (dk < p.tol) {
          status = kStatusOk;
          next = kStop;
        } else if (k >= p.max_iter) {
          status = kStatusNotConverged;
          next = kStop;
        }
        delta = dk;
        s_next = next;
        if (!ok) s_abort = 1;
      }
    }
    __syncthreads();
    if (s_next != kContinue) break;
    cur ^= 1;
  }
  if (producer) {
    if (lane == 0) drain_ring(B, u);
    return;
  }
  // X^(k) is in the buffer written by the last sweep; each row is copied by the lane that wrote it.
  const double* xres = cur ? p.xa : p.xb;
  if (warp == 0 && s_abort == 0) {
    for (int64_t g0 = r0; g0 < r1; g0 += kRows)
      if (g0 + lane < r1 && lane < kRows) p.x_out[g0 + lane] = xres[g0 + lane];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
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

// ================================================================================ IR path

// Residual phase: r_i = b_i - sum_j a_ij x_j (FP64, the full row of A), inner right-hand side
// c1_i = r_i / a_ii, first inner iterate delta^(1) = c1 (the inner iteration starts from zero).
struct ResidEpi {
  const double* b;
  const double* rinv;
  float* c1;
  float* d1;
  unsigned long long mr, mc;
  double pb, pr;
  __device__ __forceinline__ void prefetch(int64_t i) {
    pb = b[i];
    pr = rinv[i];
  }
  __device__ __forceinline__ void row(int64_t i, double dot) {
    const double r = pb - dot;
    const float c = static_cast<float>(r * pr);
    c1[i] = c;
    d1[i] = c;
    mr = umax(mr, abs_bits(r));
    mc = umax(mc, abs_bits(c));
  }
};

// Inner sweep on the narrow matrix: delta^(m)_i = c1_i - f_i * sum_j n_ij delta^(m-1)_j (the Section 2
// update of A delta = r with the stored factor f_i = 1/a_ii (times the E4M3 row scale)), plus the
// candidate X + delta^(m) in FP64, used if this is the last inner sweep of the outer step (with its
// two FP32 words when the residual is split-float).
struct InnerEpi {
  const float* c1;
  const float* rowfac;
  const double* rinv;  // fused first sweep: the factor is fl32(1/a_ii), written to rowfac_out
  float* rowfac_out;
  const float* dc;
  float* dn;
  const double* xc;
  double* xalt;
  float2* xsalt;
  int g;  // the split words are of x 2^-g
  unsigned long long mchg, mmag;
  float pc, pf, pd;
  double px;
  __device__ __forceinline__ void prefetch(int64_t i) {
    pc = c1[i];
    if (rinv) {
      pf = __double2float_rn(rinv[i]);
      rowfac_out[i] = pf;
    } else {
      pf = rowfac[i];
    }
    pd = dc[i];
    px = xc[i];
  }
  __device__ __forceinline__ void row(int64_t i, float dot) {
    const float v = fmaf(-pf, dot, pc);
    const float old = pd;
    dn[i] = v;
    const double xn = px + static_cast<double>(v);
    xalt[i] = xn;
    if (xsalt) xsalt[i] = split_x(xn, g);
    mchg = umax(mchg, abs_bits(v - old));
    mmag = umax(mmag, abs_bits(v));
  }
};

enum Kind : int { kResid = 0, kInner = 1, kDone = 2 };

template <typename TL>
__global__ void __maxnreg__(kMaxRegs) ir_solve_kernel(SolveParams p) {
  // E4M3 rows need their row scale before any entry is encoded, so that copy is always written by setup
  constexpr bool kFusable = !std::is_same<TL, __nv_fp8_e4m3>::value;
  extern __shared__ unsigned char smem_raw[];
  __shared__ Ring ring;
  __shared__ double red64[2][kConsumerWarps][kRowsPerWarp];
  __shared__ float red32[2][kConsumerWarps][kRowsPerWarp];
  __shared__ int s_abort, s_kind, s_xcur, s_dcur, s_first, s_fuse;
  char* stages = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));

  const int G = gridDim.x;
  const int64_t r0 = p.n * blockIdx.x / G, r1 = p.n * (blockIdx.x + 1) / G;
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0) p.ctl->t_start = global_timer_ns();
    s_abort = 0;
    s_kind = kResid;
    s_xcur = 0;
    s_dcur = 0;
    s_first = 1;
    // the narrow copy is still to be written: the first inner sweep writes it (every CTA reads the flag
    // here, before the grid barrier that precedes CTA 0's update of it)
    s_fuse = kFusable && p.nready != nullptr && *reinterpret_cast<volatile const int*>(p.nready) == 0;
  }
  init_ring(&ring);
  __syncthreads();
  Block B{&ring, stages, &s_abort, &p.ctl->status, p.wait_ns, p.test_drop_copy};
  const bool producer = threadIdx.x >= kConsumers;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TL* Nl = static_cast<const TL*>(p.Nlow);
  const int xg = p.rexp ? split_exponent(__ldg(p.cmax)) : 0;  // scale of the iterate's split words

  uint32_t u = 0;
  uint32_t phase = 0;
  // decision state (meaningful in warp 0 lane 0; identical in every CTA)
  int64_t outer = 0, inner_total = 0, inner_step = 0;
  double rho = 0.0, last_change = 0.0;
  int status = kStatusNotConverged;
  for (;; ++phase) {
    const int kind = s_kind;
    const int xcur = s_xcur, dcur = s_dcur;
    const bool skip_matrix = s_first && p.x0_zero;
    double* xc = xcur ? p.xb : p.xa;
    double* xalt = xcur ? p.xa : p.xb;
    const float2* xsc = xcur ? p.xsb : p.xsa;
    float2* xsalt = xcur ? p.xsa : p.xsb;
    float* dc = dcur ? p.db : p.da;
    float* dn = dcur ? p.da : p.db;
    unsigned long long v0 = 0, v1 = 0;
    if (kind == kResid) {
      ResidEpi epi{p.b, p.rinv, p.c1, p.da, 0ull, 0ull, 0.0, 0.0};
      if (producer) {
        if (!skip_matrix) produce_phase<double>(B, u, p.A, p.lda, p.n, r0, r1);
      } else if (p.rexp && !skip_matrix) {
        consume_phase_split(B, u, xsc, xg, p.n, r0, r1, p.rexp, red64, epi);
      } else {
        consume_phase<double>(B, u, xc, p.n, r0, r1, !skip_matrix, red64, epi);
      }
      v0 = epi.mr;
      v1 = epi.mc;
    } else if (s_fuse) {
      if constexpr (kFusable) {
        InnerEpi epi{p.c1, p.rowfac, p.rinv, p.rowfac_w, dc, dn, xc, xalt, p.rexp ? xsalt : nullptr, xg, 0ull, 0ull,
                     0.f, 0.f, 0.f, 0.0};
        if (producer) {
          produce_phase<double>(B, u, p.A, p.lda, p.n, r0, r1);
        } else {
          consume_phase_narrow<TL>(B, u, dc, p.n, r0, r1, static_cast<TL*>(p.Nlow_w), p.ldn, red32, epi);
        }
        v0 = epi.mchg;
        v1 = epi.mmag;
      }
    } else {
      InnerEpi epi{p.c1, p.rowfac, nullptr, nullptr, dc, dn, xc, xalt, p.rexp ? xsalt : nullptr, xg, 0ull, 0ull,
                   0.f, 0.f, 0.f, 0.0};
      if (producer) {
        produce_phase<TL>(B, u, Nl, p.ldn, p.n, r0, r1);
      } else {
        consume_phase<TL>(B, u, dc, p.n, r0, r1, true, red32, epi);
      }
      v0 = epi.mchg;
      v1 = epi.mmag;
    }
    __syncthreads();
    if (warp == 0) {
      v0 = warp_max_u64(v0);
      v1 = warp_max_u64(v1);
      int ok = 1;
      if (lane == 0) ok = (s_abort == 0) && publish_and_sync(p.ctl, phase, v0, v1, p.wait_ns);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (lane == 0) {
        trace_phase(p.ctl, phase,
                    kind == kInner ? (s_fuse ? JACOBI_PHASE_NARROW_INNER : JACOBI_PHASE_INNER)
                                   : (skip_matrix ? JACOBI_PHASE_RESID0 : JACOBI_PHASE_RESID64));
        const double g0v = bits_to_double(ld_cg_u64(&p.ctl->red[phase % 3][0]));
        const double g1v = bits_to_double(ld_cg_u64(&p.ctl->red[phase % 3][1]));
        int next = kDone;
        if (!ok) {
          status = kStatusTimeout;
          s_abort = 1;
        } else if (kind == kResid) {
          ++outer;
          rho = g0v / __ldg(p.bnorm);
          if (!isfinite(rho)) {
            status = kStatusNonfinite;
          } else if (rho <= p.tol) {
            status = kStatusOk;
          } else if (outer >= p.max_outer || inner_total >= p.max_iter) {
            status = kStatusNotConverged;
          } else {
            next = kInner;
            inner_step = 0;
            s_dcur = 0;  // delta^(1) was written into da
          }
        } else {
          if (s_fuse) {  // every CTA passed the barrier after writing its rows of the narrow copy
            s_fuse = 0;
            if (blockIdx.x == 0) *reinterpret_cast<volatile int*>(p.nready) = 1;
          }
          ++inner_total;
          ++inner_step;
          last_change = g0v;
          if (!isfinite(g0v) || !isfinite(g1v)) {
            status = kStatusNonfinite;
          } else if (g0v <= static_cast<double>(p.inner_rtol) * g1v || inner_step >= p.max_inner ||
                     inner_total >= p.max_iter) {
            next = kResid;
            s_xcur = xcur ^ 1;  // X + delta becomes the current iterate
          } else {
            next = kInner;
            s_dcur = dcur ^ 1;
          }
        }
        s_kind = next;
        s_first = 0;
      }
    }
    __syncthreads();
    if (s_kind == kDone) break;
  }
  if (producer) {
    if (lane == 0) drain_ring(B, u);
    return;
  }
  const double* xres = s_xcur ? p.xb : p.xa;
  if (warp == 0 && s_abort == 0) {
    for (int64_t g0 = r0; g0 < r1; g0 += kRows)
      if (g0 + lane < r1 && lane < kRows) p.x_out[g0 + lane] = xres[g0 + lane];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    jacobi_stats st;
    st.sweeps = inner_total;
    st.outer_steps = outer;
    st.final_delta = last_change;
    st.rel_residual = rho;
    st.status = status;
    st.converged = status == kStatusOk;
    p.ctl->result = st;
    if (p.stats_out) *p.stats_out = st;
  }
}

template <typename K>
cudaError_t launch_coop(K kernel, const SolveParams& p, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
  if (e != cudaSuccess) return e;
  SolveParams copy = p;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kernel), dim3(grid), dim3(kThreads), args,
                                     kDynSmem, s);
}

template <typename K>
int coresident(K kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, kDynSmem) != cudaSuccess) return 0;
  return per_sm * sms;
}

}  // namespace

cudaError_t launch_fp64_solve(const SolveParams& p, int grid, cudaStream_t s) {
  return launch_coop(fp64_solve_kernel, p, grid, s);
}

cudaError_t launch_ir_solve(Narrow kind, const SolveParams& p, int grid, cudaStream_t s) {
  switch (kind) {
    case Narrow::F32: return launch_coop(ir_solve_kernel<float>, p, grid, s);
    case Narrow::BF16: return launch_coop(ir_solve_kernel<__nv_bfloat16>, p, grid, s);
    case Narrow::E4M3: return launch_coop(ir_solve_kernel<__nv_fp8_e4m3>, p, grid, s);
  }
  return cudaErrorInvalidValue;
}

int max_coresident_grid(bool ir, Narrow kind) {
  if (!ir) return coresident(fp64_solve_kernel);
  switch (kind) {
    case Narrow::F32: return coresident(ir_solve_kernel<float>);
    case Narrow::BF16: return coresident(ir_solve_kernel<__nv_bfloat16>);
    case Narrow::E4M3: return coresident(ir_solve_kernel<__nv_fp8_e4m3>);
  }
  return 0;
}

}  // namespace jac
