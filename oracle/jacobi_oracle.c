/*
 * Plain FP64 CPU oracle for the dense Jacobi solver of Margaris, Souravlas & Roumeliotis,
 * "Parallel Implementations of the Jacobi Linear Algebraic Systems Solver" (arXiv:1403.5805).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code, header, table or helper with the CUDA path and is
 * deliberately slow and obvious: straight loops in the order the paper states them, no blocking, no
 * vectorisation tricks, ascending-index summation.
 *
 * Conventions (the same as the C-ABI of the CUDA library, restated here on purpose):
 *   A  row-major n x n, element (i, j) at A[i*n + j]          (Section 2: alpha_ij, row i)
 *   B, X column-major n x nrhs, element (i, c) at B[c*n + i]  (one right-hand side per column)
 *
 * Status codes: 0 converged, 1 iteration cap reached, -1 invalid argument, -2 zero diagonal entry,
 * -3 non-finite value, -4 out of memory.
 *
 * Pins of every function are in tests/test_oracle.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_INVALID_ARG (-1)
#define OR_ZERO_DIAGONAL (-2)
#define OR_NONFINITE (-3)
#define OR_NO_MEMORY (-4)

/* Stopping norms of the difference between consecutive iterates.
 *   0: max-norm, max_{i,c} |x_ic^(k) - x_ic^(k-1)|
 *   1: Euclidean norm (the paper's test, Section 2 and Eq. of Section 3.1), per right-hand side, max over
 *      right-hand sides
 *   2: relative residual of the previous iterate, max_c ( max_i |a_ii (x_ic^(k) - x_ic^(k-1))| /
 *      max_i |b_ic| ), which equals ||B - A X^(k-1)||_inf / ||B||_inf because
 *      a_ii (x_i^(k) - x_i^(k-1)) = b_i - sum_j a_ij x_j^(k-1)  (Section 2 component update). */
#define OR_NORM_INF 0
#define OR_NORM_2 1
#define OR_NORM_RESID 2

static double or_norm_of_change(int64_t n, int64_t nrhs, const double* A, const double* B,
                                const double* Xnew, const double* Xold, int norm) {
  double worst = 0.0;
  for (int64_t c = 0; c < nrhs; ++c) {
    double acc = 0.0, bmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double diff = Xnew[c * n + i] - Xold[c * n + i];
      if (norm == OR_NORM_INF) {
        double a = fabs(diff);
        if (!(a <= acc)) acc = a; /* NaN propagates */
      } else if (norm == OR_NORM_2) {
        acc += diff * diff;
      } else {
        double a = fabs(A[i * n + i] * diff);
        if (!(a <= acc)) acc = a;
        double b = fabs(B[c * n + i]);
        if (b > bmax) bmax = b;
      }
    }
    if (norm == OR_NORM_2) acc = sqrt(acc);
    if (norm == OR_NORM_RESID) acc = acc / bmax; /* ||b|| = 0 gives inf or NaN: reported as non-finite */
    if (!(acc <= worst)) worst = acc;
  }
  return worst;
}

/*
 * Jacobi iteration, Section 2.
 *   x_i^(k) = ( beta_i - sum_{j != i} alpha_ij x_j^(k-1) ) / alpha_ii     (Section 2 component update)
 * with the control flow of the Section 2 serial algorithm: k runs from 1 to L; after each sweep the
 * change between consecutive iterates is measured and, if it is below tol (strict), the new iterate is
 * returned; otherwise the new iterate becomes the old one.  If L sweeps pass without meeting the test,
 * X^(L) is returned with status 1.
 *
 * X0 may be NULL (zeros).  trace, if not NULL, receives X^(k) for k = 1..iters at trace[(k-1)*n*nrhs].
 * nthreads > 1 splits the rows of each sweep over OpenMP threads (the paper's row-wise distribution of
 * Section 3.1, on shared memory); results do not depend on it.
 */
int oracle_jacobi(int64_t n, int64_t nrhs, const double* A, const double* B, const double* X0,
                  int64_t max_iter, double tol, int norm, int nthreads, double* X_out,
                  int64_t* iters_out, double* delta_out, double* trace) {
  if (n < 1 || nrhs < 1 || !A || !B || !X_out || !iters_out || !delta_out) return OR_INVALID_ARG;
  if (max_iter < 1 || !(tol > 0.0) || norm < 0 || norm > 2) return OR_INVALID_ARG;
  /* The method needs alpha_ii != 0 (Section 2). */
  for (int64_t i = 0; i < n; ++i) {
    double d = A[i * n + i];
    if (!isfinite(d)) return OR_NONFINITE;
    if (d == 0.0) return OR_ZERO_DIAGONAL;
  }
  size_t len = (size_t)n * (size_t)nrhs;
  double* Xt = (double*)malloc(len * sizeof(double));
  double* X = (double*)malloc(len * sizeof(double));
  if (!Xt || !X) {
    free(Xt);
    free(X);
    return OR_NO_MEMORY;
  }
  if (X0)
    memcpy(Xt, X0, len * sizeof(double));
  else
    memset(Xt, 0, len * sizeof(double));
  if (nthreads < 1) nthreads = 1;

  int status = OR_NOT_CONVERGED;
  int64_t k;
  double delta = 0.0;
  for (k = 1; k <= max_iter; ++k) {
    /* one sweep: every component from the previous iterate only */
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t c = 0; c < nrhs; ++c) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
          if (j == i) continue;
          s += A[i * n + j] * Xt[c * n + j];
        }
        X[c * n + i] = (B[c * n + i] - s) / A[i * n + i];
      }
    }
    if (trace) memcpy(trace + (size_t)(k - 1) * len, X, len * sizeof(double));
    delta = or_norm_of_change(n, nrhs, A, B, X, Xt, norm);
    if (!isfinite(delta)) {
      status = OR_NONFINITE;
      memcpy(X_out, X, len * sizeof(double));
      break;
    }
    if (delta < tol) {
      status = OR_OK;
      memcpy(X_out, X, len * sizeof(double));
      break;
    }
    /* X^t = X */
    double* tmp = Xt;
    Xt = X;
    X = tmp;
  }
  if (status == OR_NOT_CONVERGED) {
    k = max_iter;
    memcpy(X_out, Xt, len * sizeof(double)); /* X^(L) */
  }
  *iters_out = k;
  *delta_out = delta;
  free(Xt);
  free(X);
  return status;
}

/*
 * Block-hybrid Gauss-Seidel / SOR, the relaxed relative of the Section 2 iteration that the paper's
 * introduction lists among the iterative solvers, in the row-blocked form a parallel machine runs:
 * the unknowns are split into consecutive row blocks [s_b, s_(b+1)); inside a block the components
 * are updated in ascending order using the block's newest values, across blocks using the previous
 * iterate, and each update is relaxed by omega:
 *   v_i     = ( beta_i - sum_{j != i} alpha_ij xt_j ) / alpha_ii,
 *             xt_j = x_j^(k) if s_b <= j < i (same block, already updated), else x_j^(k-1)
 *   x_i^(k) = v_i                                  if omega == 1 (Gauss-Seidel inside blocks)
 *           = x_i^(k-1) + omega (v_i - x_i^(k-1))  otherwise.
 * One block per row with omega = 1 is exactly the Jacobi iteration above; a single block is classical
 * SOR (Gauss-Seidel for omega = 1).  The control flow, the stopping test (strict, on the change between
 * consecutive iterates, norm 0 or 1 of oracle_jacobi) and the return conventions are those of
 * oracle_jacobi.  block_start holds nblocks + 1 ascending offsets from 0 to n.
 */
int oracle_block_sor(int64_t n, int64_t nrhs, const double* A, const double* B, const double* X0,
                     int64_t max_iter, double tol, int norm, int64_t nblocks, const int64_t* block_start,
                     double omega, double* X_out, int64_t* iters_out, double* delta_out, double* trace) {
  if (n < 1 || nrhs < 1 || !A || !B || !X_out || !iters_out || !delta_out || !block_start) return OR_INVALID_ARG;
  if (max_iter < 1 || !(tol > 0.0) || (norm != OR_NORM_INF && norm != OR_NORM_2)) return OR_INVALID_ARG;
  if (nblocks < 1 || block_start[0] != 0 || block_start[nblocks] != n) return OR_INVALID_ARG;
  for (int64_t b = 0; b < nblocks; ++b)
    if (block_start[b + 1] < block_start[b]) return OR_INVALID_ARG;
  if (!(omega > 0.0 && omega < 2.0)) return OR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i) {
    double d = A[i * n + i];
    if (!isfinite(d)) return OR_NONFINITE;
    if (d == 0.0) return OR_ZERO_DIAGONAL;
  }
  size_t len = (size_t)n * (size_t)nrhs;
  double* Xt = (double*)malloc(len * sizeof(double));
  double* X = (double*)malloc(len * sizeof(double));
  if (!Xt || !X) {
    free(Xt);
    free(X);
    return OR_NO_MEMORY;
  }
  if (X0)
    memcpy(Xt, X0, len * sizeof(double));
  else
    memset(Xt, 0, len * sizeof(double));

  int status = OR_NOT_CONVERGED;
  int64_t k;
  double delta = 0.0;
  for (k = 1; k <= max_iter; ++k) {
    for (int64_t b = 0; b < nblocks; ++b) {
      const int64_t s0 = block_start[b], s1 = block_start[b + 1];
      for (int64_t i = s0; i < s1; ++i) {
        for (int64_t c = 0; c < nrhs; ++c) {
          double s = 0.0;
          for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double xj = (j >= s0 && j < i) ? X[c * n + j] : Xt[c * n + j];
            s += A[i * n + j] * xj;
          }
          const double v = (B[c * n + i] - s) / A[i * n + i];
          X[c * n + i] = omega == 1.0 ? v : Xt[c * n + i] + omega * (v - Xt[c * n + i]);
        }
      }
    }
    if (trace) memcpy(trace + (size_t)(k - 1) * len, X, len * sizeof(double));
    delta = or_norm_of_change(n, nrhs, A, B, X, Xt, norm);
    if (!isfinite(delta)) {
      status = OR_NONFINITE;
      memcpy(X_out, X, len * sizeof(double));
      break;
    }
    if (delta < tol) {
      status = OR_OK;
      memcpy(X_out, X, len * sizeof(double));
      break;
    }
    double* tmp = Xt;
    Xt = X;
    X = tmp;
  }
  if (status == OR_NOT_CONVERGED) {
    k = max_iter;
    memcpy(X_out, Xt, len * sizeof(double));
  }
  *iters_out = k;
  *delta_out = delta;
  free(Xt);
  free(X);
  return status;
}

/*
 * Jacobi iteration for a sparse A stored in compressed sparse rows: the same Section 2 component update
 * and control flow as oracle_jacobi, with the sum running over the stored entries of row i only:
 *   x_i^(k) = ( beta_i - sum_{stored j != i} alpha_ij x_j^(k-1) ) / alpha_ii.
 * Row i holds col_idx[row_ptr[i] .. row_ptr[i+1]) (strictly ascending, so the sum runs in ascending j as
 * in oracle_jacobi) and the matching values; its diagonal must be among them.  One right-hand side;
 * stopping norm 0 (max), 1 (Euclidean) or 2 (relative residual of the previous iterate, as oracle_jacobi).  Validation, in this order: the CSR structure (row_ptr starts
 * at 0 and never decreases, columns in range and strictly ascending) -> -1; then, row by row, a missing or
 * zero diagonal -> -2, a non-finite one -> -3.
 */
int oracle_csr_jacobi(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                      const double* B, const double* X0, int64_t max_iter, double tol, int norm, double* X_out,
                      int64_t* iters_out, double* delta_out, double* trace) {
  if (n < 1 || !row_ptr || !B || !X_out || !iters_out || !delta_out) return OR_INVALID_ARG;
  if (max_iter < 1 || !(tol > 0.0) || norm < OR_NORM_INF || norm > OR_NORM_RESID) return OR_INVALID_ARG;
  if (row_ptr[0] != 0) return OR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) return OR_INVALID_ARG;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      if (col_idx[e] < 0 || col_idx[e] >= n) return OR_INVALID_ARG;
      if (e > row_ptr[i] && col_idx[e] <= col_idx[e - 1]) return OR_INVALID_ARG;
    }
  }
  double* diag = (double*)malloc((size_t)n * sizeof(double));
  double* Xt = (double*)malloc((size_t)n * sizeof(double));
  double* X = (double*)malloc((size_t)n * sizeof(double));
  if (!diag || !Xt || !X) {
    free(diag);
    free(Xt);
    free(X);
    return OR_NO_MEMORY;
  }
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      if (col_idx[e] == i) d = val[e];
    if (!isfinite(d)) {
      free(diag);
      free(Xt);
      free(X);
      return OR_NONFINITE;
    }
    if (d == 0.0) {
      free(diag);
      free(Xt);
      free(X);
      return OR_ZERO_DIAGONAL;
    }
    diag[i] = d;
  }
  if (X0)
    memcpy(Xt, X0, (size_t)n * sizeof(double));
  else
    memset(Xt, 0, (size_t)n * sizeof(double));

  int status = OR_NOT_CONVERGED;
  int64_t k;
  double delta = 0.0;
  for (k = 1; k <= max_iter; ++k) {
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        if (col_idx[e] == i) continue;
        s += val[e] * Xt[col_idx[e]];
      }
      X[i] = (B[i] - s) / diag[i];
    }
    if (trace) memcpy(trace + (size_t)(k - 1) * (size_t)n, X, (size_t)n * sizeof(double));
    if (norm == OR_NORM_RESID) { /* max_i |a_ii (x_i^(k) - x_i^(k-1))| / max_i |b_i|, as or_norm_of_change */
      double acc = 0.0, bmax = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        double a = fabs(diag[i] * (X[i] - Xt[i]));
        if (!(a <= acc)) acc = a;
        if (fabs(B[i]) > bmax) bmax = fabs(B[i]);
      }
      delta = acc / bmax;
    } else {
      delta = or_norm_of_change(n, 1, NULL, B, X, Xt, norm);
    }
    if (!isfinite(delta)) {
      status = OR_NONFINITE;
      memcpy(X_out, X, (size_t)n * sizeof(double));
      break;
    }
    if (delta < tol) {
      status = OR_OK;
      memcpy(X_out, X, (size_t)n * sizeof(double));
      break;
    }
    double* tmp = Xt;
    Xt = X;
    X = tmp;
  }
  if (status == OR_NOT_CONVERGED) {
    k = max_iter;
    memcpy(X_out, Xt, (size_t)n * sizeof(double));
  }
  *iters_out = k;
  *delta_out = delta;
  free(diag);
  free(Xt);
  free(X);
  return status;
}

/*
 * Gaussian elimination with partial (row) pivoting, then back substitution: the textbook direct
 * solver used to pin the converged Jacobi value on small systems.  Returns -2 on an exactly zero pivot.
 */
int oracle_ge(int64_t n, int64_t nrhs, const double* A, const double* B, double* X) {
  if (n < 1 || nrhs < 1 || !A || !B || !X) return OR_INVALID_ARG;
  double* M = (double*)malloc((size_t)n * n * sizeof(double));
  double* R = (double*)malloc((size_t)n * nrhs * sizeof(double));
  if (!M || !R) {
    free(M);
    free(R);
    return OR_NO_MEMORY;
  }
  memcpy(M, A, (size_t)n * n * sizeof(double));
  /* R is row-major n x nrhs so that a row swap moves one contiguous row */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t c = 0; c < nrhs; ++c) R[i * nrhs + c] = B[c * n + i];
  int status = OR_OK;
  for (int64_t p = 0; p < n && status == OR_OK; ++p) {
    int64_t piv = p;
    for (int64_t i = p + 1; i < n; ++i)
      if (fabs(M[i * n + p]) > fabs(M[piv * n + p])) piv = i;
    if (M[piv * n + p] == 0.0) {
      status = OR_ZERO_DIAGONAL;
      break;
    }
    if (piv != p) {
      for (int64_t j = 0; j < n; ++j) {
        double t = M[p * n + j];
        M[p * n + j] = M[piv * n + j];
        M[piv * n + j] = t;
      }
      for (int64_t c = 0; c < nrhs; ++c) {
        double t = R[p * nrhs + c];
        R[p * nrhs + c] = R[piv * nrhs + c];
        R[piv * nrhs + c] = t;
      }
    }
    for (int64_t i = p + 1; i < n; ++i) {
      double l = M[i * n + p] / M[p * n + p];
      for (int64_t j = p; j < n; ++j) M[i * n + j] -= l * M[p * n + j];
      for (int64_t c = 0; c < nrhs; ++c) R[i * nrhs + c] -= l * R[p * nrhs + c];
    }
  }
  if (status == OR_OK) {
    for (int64_t c = 0; c < nrhs; ++c) {
      for (int64_t i = n - 1; i >= 0; --i) {
        double s = R[i * nrhs + c];
        for (int64_t j = i + 1; j < n; ++j) s -= M[i * n + j] * X[c * n + j];
        X[c * n + i] = s / M[i * n + i];
      }
    }
  }
  free(M);
  free(R);
  return status;
}

/*
 * Residual R = B - A X in FP64 (ascending-index sums), and the relative residual
 * max_c ||r_c||_inf / ||b_c||_inf, the stopping quantity of the mixed-precision refinement.
 * R may be NULL.
 */
int oracle_residual(int64_t n, int64_t nrhs, const double* A, const double* B, const double* X,
                    double* R, double* rel_out) {
  if (n < 1 || nrhs < 1 || !A || !B || !X || !rel_out) return OR_INVALID_ARG;
  double worst = 0.0;
  for (int64_t c = 0; c < nrhs; ++c) {
    double rmax = 0.0, bmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += A[i * n + j] * X[c * n + j];
      double r = B[c * n + i] - s;
      if (R) R[c * n + i] = r;
      if (!(fabs(r) <= rmax)) rmax = fabs(r);
      if (fabs(B[c * n + i]) > bmax) bmax = fabs(B[c * n + i]);
    }
    double rel = rmax / bmax;
    if (!(rel <= worst)) worst = rel;
  }
  *rel_out = worst;
  return OR_OK;
}

/*
 * The residual of oracle_residual restricted to the listed rows: R[c * nrows + t] = b_ic - sum_j a_ij x_jc
 * for i = rows[t], with the same ascending-j sum per row, for checking large systems on a sample of rows.
 */
int oracle_residual_rows(int64_t n, int64_t nrhs, const double* A, const double* B, const double* X,
                         int64_t nrows, const int64_t* rows, double* R) {
  if (n < 1 || nrhs < 1 || nrows < 0 || !A || !B || !X || !R || (nrows > 0 && !rows)) return OR_INVALID_ARG;
  for (int64_t t = 0; t < nrows; ++t)
    if (rows[t] < 0 || rows[t] >= n) return OR_INVALID_ARG;
  for (int64_t c = 0; c < nrhs; ++c) {
    for (int64_t t = 0; t < nrows; ++t) {
      int64_t i = rows[t];
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += A[i * n + j] * X[c * n + j];
      R[c * nrows + t] = B[c * n + i] - s;
    }
  }
  return OR_OK;
}

/*
 * Residual r = b - A x of a CSR matrix in FP64 (the stored entries of each row in their ascending column
 * order, the diagonal included), and the relative residual ||r||_inf / ||b||_inf.  r may be NULL.  The
 * structure is trusted (oracle_csr_jacobi checks it).
 */
int oracle_csr_residual(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                        const double* B, const double* X, double* R, double* rel_out) {
  if (n < 1 || !row_ptr || !B || !X || !rel_out) return OR_INVALID_ARG;
  double rmax = 0.0, bmax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += val[e] * X[col_idx[e]];
    double r = B[i] - s;
    if (R) R[i] = r;
    if (!(fabs(r) <= rmax)) rmax = fabs(r);
    if (fabs(B[i]) > bmax) bmax = fabs(B[i]);
  }
  *rel_out = rmax / bmax;
  return OR_OK;
}

/*
 * Fixed-point form of Section 2: A = D - L - U, X = T X + C with T = D^-1 (L + U), C = D^-1 B.
 * With L and U the negated strict triangles of A this is t_ij = -alpha_ij / alpha_ii (j != i),
 * t_ii = 0, c_i = beta_i / alpha_ii, each a single correctly rounded IEEE division.
 * T is row-major n x n, C column-major n x nrhs.
 */
int oracle_split(int64_t n, int64_t nrhs, const double* A, const double* B, double* T, double* C) {
  if (n < 1 || nrhs < 1 || !A || !B || !T || !C) return OR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i) {
    double d = A[i * n + i];
    if (!isfinite(d)) return OR_NONFINITE;
    if (d == 0.0) return OR_ZERO_DIAGONAL;
  }
  for (int64_t i = 0; i < n; ++i) {
    double d = A[i * n + i];
    for (int64_t j = 0; j < n; ++j) T[i * n + j] = (j == i) ? 0.0 : -A[i * n + j] / d;
    for (int64_t c = 0; c < nrhs; ++c) C[c * n + i] = B[c * n + i] / d;
  }
  return OR_OK;
}

/* ---- low-precision storage for the inner sweeps of the mixed-precision refinement -------------------
 * Section 2 writes T = D^-1 (L + U): the off-diagonal part of A scaled row by row by 1/alpha_ii.  The
 * narrow copies keep that factorisation: they store the off-diagonal entries alpha_ij (j != i, zero on
 * the diagonal) in a narrow type and leave the row factor 1/alpha_ii (and, for E4M3, a row scale) in
 * full precision.  Reading adopted for every type: alpha_ij is first rounded to FP32 (round to nearest
 * even, the C cast), then
 *   FP32:     kept as is;
 *   BF16:     rounded to nearest even into BF16 (sign, 8 exponent bits, 7 fraction bits);
 *   FP8 E4M3: per-row scale s_i = the smallest power of two 2^k (-126 <= k <= 127) with
 *             max_{j != i} |a32_ij| <= 448 s_i (448 is the largest finite E4M3 value), s_i = 1 when the
 *             maximum is 0; code q_ij = E4M3 value nearest to a32_ij / s_i (FP32 division, exact for a
 *             power of two), ties to the code with an even last mantissa bit, saturating to +-448.  A
 *             power-of-two scale leaves every entry's relative rounding error what it would be unscaled.
 * Both encoders below work from the formats' definitions (value tables), not from bit tricks. */

static float or_bf16_value(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

/* BF16 is exactly the upper half of an FP32 encoding.  The nearest BF16 of a finite FP32 x is one of
 * two candidates: x's encoding truncated, or that truncation stepped one unit away from zero.  Pick
 * the nearer; on a tie the one whose last bit is even. */
uint16_t oracle_bf16_from_f32(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if (isnan(x)) return (uint16_t)((u >> 16) | 0x0040u); /* quiet NaN, sign kept */
  uint16_t lo = (uint16_t)(u >> 16);
  if ((u & 0xFFFFu) == 0) return lo; /* exactly representable */
  uint16_t hi = (uint16_t)(lo + 1);  /* next encoding away from zero (may reach infinity) */
  double dx = fabs((double)x);
  /* IEEE rounding measures the step past the largest finite value as if the exponent range were
   * unbounded: the infinity encoding stands for 2^128 here */
  double vhi = ((hi & 0x7FFFu) == 0x7F80u) ? ldexp(1.0, 128) : fabs((double)or_bf16_value(hi));
  double elo = dx - fabs((double)or_bf16_value(lo)); /* both differences exact in FP64 */
  double ehi = vhi - dx;
  if (elo < ehi) return lo;
  if (ehi < elo) return hi;
  return (lo & 1u) ? hi : lo;
}

/* E4M3 (the "fn" variant: no infinities, S.1111.111 is NaN): value of a code. */
static double or_e4m3_value(uint8_t q) {
  int s = (q >> 7) & 1, e = (q >> 3) & 0xF, m = q & 7;
  double v = (e == 0) ? ldexp((double)m / 8.0, -6) : ldexp(1.0 + (double)m / 8.0, e - 7);
  return s ? -v : v;
}

/* Nearest E4M3 code of x, ties to even mantissa, saturating to the largest finite magnitude. */
uint8_t oracle_e4m3_from_f32(float x) {
  if (isnan(x)) return 0x7F;
  uint8_t sign = signbit(x) ? 0x80 : 0x00;
  double a = fabs((double)x);
  if (a >= or_e4m3_value(0x7E)) return (uint8_t)(sign | 0x7E);
  /* the 127 non-negative finite codes 0x00..0x7E increase with the code: find the largest code whose
   * value is <= a by binary search, then compare with its successor */
  int lo = 0, hi = 0x7E;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (or_e4m3_value((uint8_t)mid) <= a)
      lo = mid;
    else
      hi = mid - 1;
  }
  int below = lo, above = lo + 1;
  double eb = a - or_e4m3_value((uint8_t)below), ea = or_e4m3_value((uint8_t)above) - a;
  int pick;
  if (eb < ea)
    pick = below;
  else if (ea < eb)
    pick = above;
  else
    pick = (below & 1) ? above : below;
  return (uint8_t)(sign | pick);
}

/* Off-diagonal part of A (row-major n x n) in FP32, zero on the diagonal. */
void oracle_offdiag_f32(int64_t n, const double* A, float* out) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) out[i * n + j] = (j == i) ? 0.0f : (float)A[i * n + j];
}

/* Off-diagonal part of A in BF16 codes (through FP32), zero on the diagonal. */
void oracle_offdiag_bf16(int64_t n, const double* A, uint16_t* out) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      out[i * n + j] = (j == i) ? (uint16_t)0 : oracle_bf16_from_f32((float)A[i * n + j]);
}

/* The E4M3 row scale: smallest power of two 2^k, -126 <= k <= 127, with m <= 448 * 2^k (1 for m = 0). */
static float or_e4m3_row_scale(float m) {
  if (m == 0.0f) return 1.0f;
  int k = -126;
  if (!isfinite(m))
    k = 127;
  else
    while (k < 127 && (double)m > 448.0 * ldexp(1.0, k)) ++k;
  return ldexpf(1.0f, k);
}

/* Off-diagonal part of A as per-row scaled E4M3 codes (through FP32), zero code on the diagonal. */
void oracle_offdiag_e4m3(int64_t n, const double* A, uint8_t* q, float* scale) {
  for (int64_t i = 0; i < n; ++i) {
    float m = 0.0f;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      float a = fabsf((float)A[i * n + j]);
      if (a > m) m = a;
    }
    float s = or_e4m3_row_scale(m);
    scale[i] = s;
    for (int64_t j = 0; j < n; ++j)
      q[i * n + j] = (j == i) ? (uint8_t)0 : oracle_e4m3_from_f32((float)A[i * n + j] / s);
  }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
