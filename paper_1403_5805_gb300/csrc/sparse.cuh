// Sparse (CSR input) Jacobi solve (sparse.cu): declarations shared with the host layer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "solver.cuh"

namespace jac {

constexpr int kSliceRows = 32;  // rows per slice of the sliced-ELL copy: one warp, one row per lane
constexpr int kMaxDiag = 16;    // most diagonals of the DIA copy (more, or a poorly filled band: sliced ELL)

// Setup pass 1 (one thread per row) over CSR arrays in device memory: checks the structure and the
// diagonal, writes d_i = a_ii and the row's off-diagonal count.  The first failure by the oracle's order is
// left in *key (all ones beforehand) as (class << 56) | (row << 8) | code: class 0 = structure (code 1:
// row_ptr[0] != 0, a row range that decreases or leaves [0, nnz), a column out of range, or columns not
// strictly ascending), class 1 = diagonal (code 2: missing or zero, code 3: non-finite).  Only entries
// inside [0, nnz) are read.
cudaError_t launch_csr_check(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                             const double* val, double* d, int32_t* lens, unsigned long long* key, cudaStream_t s);
// Setup pass 2: width[s] = max off-diagonal count over the rows of slice s (one warp per slice).
cudaError_t launch_csr_widths(int64_t n, const int32_t* lens, int32_t* width, cudaStream_t s);
// Setup pass 3: T = D^-1 (L + U) as a sliced-ELL copy, t_ij = -a_ij / a_ii, and C = D^-1 B in place
// (c holds b on entry); *bmax (zero beforehand) receives the IEEE bits of ||b||_inf.  Entry t of row i = 32 s + l sits at soff[s] + 32 t + l (column-major inside the
// slice, so a warp's loads of one entry index are one 256-byte run); slots past the row's length hold
// value 0 and the column min(i, n - 1).
cudaError_t launch_csr_fill(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                            const double* d, const int64_t* soff, double* sval, int32_t* scol, double* c,
                            unsigned long long* bmax, cudaStream_t s);
// DIA alternative to pass 3 for banded and stencil matrices: *bad (zero beforehand) becomes nonzero if
// some off-diagonal entry's offset j - i is not among doff[0..ndiag); the fill writes entry t of row i at
// dval[((i / 32) * ndiag + t) * 32 + i % 32] (dval zero beforehand, ndiag times n rounded up to whole
// slices), and C as pass 3 does.
cudaError_t launch_csr_dia_check(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const int32_t* doff,
                                 int ndiag, int* bad, cudaStream_t s);
cudaError_t launch_csr_dia_fill(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                                const double* d, const int32_t* doff, int ndiag, double* dval, double* c,
                                unsigned long long* bmax, cudaStream_t s);

struct CsrParams {
  int64_t n, nslices;
  const int64_t* soff;  // nslices + 1 slot offsets (multiples of 32)
  const double* sval;   // t_ij = -a_ij / a_ii, sliced ELL
  const int32_t* scol;  // their columns
  const double* c;      // c_i = b_i / a_ii
  double* xa;           // iterate buffers (length 32 nslices, zero past n): x^(0) in xa, then alternating
  double* xb;
  double* part;         // [2][kMaxGrid] per-CTA partial sums (Euclidean norm)
  Ctl* ctl;             // zeroed before the launch
  double* x_out;
  jacobi_stats* stats_out;
  int64_t max_iter;
  double tol;
  int norm;             // JACOBI_NORM_INF, JACOBI_NORM_2 or JACOBI_NORM_RESID
  const double* d;      // a_ii (JACOBI_NORM_RESID)
  double bnorm;         // ||b||_inf (JACOBI_NORM_RESID)
  int test_skip_arrival;  // test only: CTA 0 skips the first grid barrier and raises the error word
  uint64_t wait_ns;
  // DIA copy (ndiag > 0): sval holds entry t of row i (column i + doff[t]) at ((i / 32) * ndiag + t) * 32
  // + i % 32, doff the ascending offsets j - i; soff and scol are unused, and xa, xb (and the FP32 vectors of the refinement) have a zero
  // halo of max |doff| entries on both sides.  ndiag == 0: sliced ELL.
  const int32_t* doff;
  int ndiag;
};

// One cooperative launch of `grid` CTAs runs the whole solve.
cudaError_t launch_csr_solve(const CsrParams& p, int grid, cudaStream_t s);

// Mixed-precision refinement of the sparse system: FP64 outer residuals r' = C + T x - x (= D^-1 (b - A x))
// with the stopping test max_i |a_ii r'_i| / ||b||_inf <= tol, inner Jacobi sweeps on the correction,
// delta <- r' + T_lo delta, with T stored in the inner type (FP32 or BF16) and FP32 accumulation, x += delta
// folded into the next residual.  `base` carries the FP64 layout, the iterates, the control block and tol.
struct CsrIrParams {
  CsrParams base;       // also a_ii and ||b||_inf (base.d, base.bnorm)
  const void* tlo;      // T in the inner type, same slots as base.sval
  float* rf;            // r' of the current outer step
  float* da;            // inner iterates
  float* db;
  float inner_rtol;     // inner stop: max |delta' - delta| <= inner_rtol * max |delta'|
  int max_inner;        // inner sweeps per outer step
  int max_outer;        // outer steps (residual evaluations after the first)
};
enum class CsrInner : int { F32 = 1, BF16 = 2 };
// T in the inner type from the FP64 slots (round to nearest).
cudaError_t launch_csr_narrow(CsrInner kind, const double* sval, int64_t slots, void* tlo, cudaStream_t s);
cudaError_t launch_csr_ir_solve(CsrInner kind, const CsrIrParams& p, int grid, cudaStream_t s);
int csr_ir_max_grid(CsrInner kind);
// Largest co-resident grid of the sweep kernel, capped at kMaxGrid (0 on failure), and its warps per CTA.
int csr_max_grid();
int csr_warps_per_cta();

}  // namespace jac
