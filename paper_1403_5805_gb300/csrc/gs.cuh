// Chained Gauss-Seidel / SOR solve (gs.cu): declarations shared with the host layer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "solver.cuh"

namespace jac {

constexpr int kGsThreads = 256;   // 8 warps per CTA
constexpr int kGsMaxRows = 112;   // rows per CTA block
constexpr int kGsPitch = kGsMaxRows + 1;  // shared-memory row pitch of the block tiles (odd: no bank clash)
// Two block tiles (the diagonal block with the inverse of its lower part; -omega M^-1 times this CTA's rows
// x the previous block's columns, as float-float pairs), five FP64 vectors, the previous block's values as
// float-float pairs and the row scale exponents of Q and of A.
constexpr size_t kGsSmem = 2 * sizeof(double) * kGsMaxRows * kGsPitch + 5 * sizeof(double) * kGsMaxRows +
                           kGsMaxRows * (sizeof(float2) + 2 * sizeof(int));

struct GsParams {
  int64_t n;
  const double* A;      // FP64 A, row-major, row stride lda
  int64_t lda;
  const double* b;
  const double* d;      // a_ii
  const double* rinv;   // 1 / a_ii
  double* xa;           // iterate buffers: x^(k-1) and x^(k) alternate
  double* xb;
  int* flags;           // one per CTA, zeroed before the launch: the last sweep whose block is final
  unsigned long long* mbox;  // [2][n] mailboxes of x^(k) (k odd / even) for the next block, all bits set before the launch
  double* part;         // [3][kMaxGrid] per-CTA partial sums (Euclidean norm), one slot per sweep mod 3
  Ctl* ctl;
  double* x_out;
  jacobi_stats* stats_out;
  int64_t max_iter;
  double tol;
  int norm;             // JACOBI_NORM_INF or JACOBI_NORM_2
  double omega;         // relaxation, 0 < omega < 2 (1: Gauss-Seidel)
  const unsigned long long* cmax;  // IEEE bits of max_i |b_i / a_ii|: the scale of the float-float split of x
  const int* rexp;      // per row: split exponent of max_j |a_ij| (launch_gs_row_exponents)
  int test_skip_publish;  // test only: block 0 never publishes sweep 1 and raises the error word
  uint64_t wait_ns;
};

// Launch on `grid` co-resident CTAs (cooperative); rows are split as r_c = n c / grid, so grid must be at
// least ceil(n / kGsMaxRows).
cudaError_t launch_gs_solve(const GsParams& p, int grid, cudaStream_t s);
// Largest co-resident grid of the kernel (0 on failure).
int gs_max_grid();
// rexp[i] = split exponent of max_j |a_ij| (|a_ij| 2^-rexp[i] < 1): the row scales of the float-float row
// products, computed once per handle.
cudaError_t launch_gs_row_exponents(const double* A, int64_t lda, int64_t n, int* rexp, cudaStream_t s);

}  // namespace jac
