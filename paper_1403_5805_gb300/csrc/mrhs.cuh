// Multi-right-hand-side kernels (mrhs.cu): the tcgen05 BF16 sweep and the FP64 dense pass.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace jac {

// Rows per block of the FP64 dense pass (mrhs_dense_kernel); its Euclidean partials are per such tile.
constexpr int kMrhsDenseRows = 32;

// One inner sweep for r right-hand sides (vectors stored v[c*ld + i]).
struct MrhsSweepParams {
  int64_t n, r, ld;
  const float* rowfac;      // n: 1 / a_ii (FP32)
  const float* c1;          // inner right-hand side D^-1 R
  const float* dc;          // previous inner iterate (FP32)
  float* dn;                // new inner iterate (FP32)
  __nv_bfloat16* dnh;       // its BF16 copy: the B operand of the next sweep
  const double* xc;         // current FP64 iterate
  double* xalt;             // xc + dn
  unsigned long long* stats;  // [0] max |dn - dc|, [1] max |dn| (IEEE bits, order-free max)
  int* status;              // set to a timeout code if a bounded wait expires
};

// FP64 pass over A for all r columns (the split-float residual when xs is set).  mode 0: residual
// R = B - A X -> c1 = R / a_ii, d1 = c1 (FP32 and BF16), colmax[c] = max_i |R_ic|.  mode 1: Jacobi sweep
// xn = (B - A x + a_ii x) / a_ii, colmax[c] = max_i |xn - x|.
struct MrhsDenseParams {
  int64_t n, r, ld, lda;
  int mode;
  int resid_norm;   // mode 1: colmax of |a_ii (xn - x)| (residual of x) instead of |xn - x|
  const double* A;
  const double* b;
  const double* x;
  const double* d;
  const double* rinv;
  float* c1;
  float* d1;
  __nv_bfloat16* d1h;
  double* xn;
  unsigned long long* colmax;
  // split-float residual (mode 0 only; NULL xs selects the FP64 pass): per-row scale exponents of A,
  // the two FP32 words of x 2^-g_c per entry, and the column exponents g_c
  const int* rexp;
  const float2* xs;
  const int* xexp;
  // active columns: tile column c works on column cols[c] (c < nact); NULL cols: all r columns
  const int* cols;
  int64_t nact;
  // mode 1, Euclidean norm: the sum of squared changes of each kMrhsDenseRows-row tile and column, written
  // (no atomics, a fixed summation order) at colsq[tile * r + c]; NULL: the maxima only
  double* colsq;
};

// FP64-accurate residual on the tensor cores (ozaki.cu): A's off-diagonal part and X split into kOzDigits
// balanced base-256 BF16 digits each; products of digit pairs summed exactly in FP32 chunks.
constexpr int kOzDigits = 7;
// Rows of each of A's digit matrices: n rounded up to the 128-row tile.
int64_t oz_padded_rows(int64_t n);

// Residual pass R = B - A X (all r columns computed; active columns written as mode 0 of the FP64 pass:
// c1 = R / a_ii, d1 = c1 (FP32, BF16), colmax[c] = max_i |R_ic|).
struct OzResidParams {
  int64_t n, r, ld, nr;
  const int* aexp;          // nr: exponent of each row's off-diagonal maximum (A's digit scale)
  const int* xexp;          // r: exponent of each column's maximum (X's digit scale)
  const double* x;          // FP64 iterate x[c*ld + i]
  const double* b;
  const double* d;          // a_ii
  const double* rinv;       // 1 / a_ii
  float* c1;
  float* d1;
  __nv_bfloat16* d1h;
  unsigned long long* colmax;
  const int* cols;          // active columns (NULL: all)
  int64_t nact;
  int* status;              // set to a timeout code if a bounded wait expires
  uint64_t wait_ns;
  // grouped launches only (launch_oz_grouped): where the X split writes X's digits and column exponents
  __nv_bfloat16* xd;
  int* xexp_w;
  // launch_oz_resid only: scratch for the K-split (kOzMaxParts x r x ld float-float partial sums); NULL
  // keeps every tile whole
  float2* part;
};
// Most parts the K range of a residual tile is split into (launch_oz_resid splits it when the row tiles
// alone would leave part of the last wave of CTAs empty).
constexpr int kOzMaxParts = 8;
// dig[(p*nr + i)*ld + j]: digit p of a_ij (j != i), zero elsewhere; aexp[i] as above.  A row-major with
// 16-byte aligned rows (lda even).
cudaError_t launch_oz_split_a(const double* A, int64_t lda, int64_t n, int64_t ld, __nv_bfloat16* dig, int* aexp,
                              cudaStream_t s);
// xd[(q*r + c)*ld + i]: digit q of x_ic; xexp[c].
cudaError_t launch_oz_split_x(int64_t n, int64_t r, int64_t ld, const double* x, __nv_bfloat16* xd, int* xexp,
                              cudaStream_t s);
cudaError_t launch_oz_resid(const __nv_bfloat16* adig, const __nv_bfloat16* xdig, const OzResidParams& p,
                            cudaStream_t s);
// Grouped residuals of requests with at most kOzServeCols right-hand sides (r <= 16): X's digits laid out
// [kOzDigits][kOzServeCols][ld] (columns >= r zero), r = kOzServeCols in the params.
constexpr int kOzServeCols = 16;
// The two tensor maps of one request (A's digits, X's digits) into maps[0], maps[1].
bool oz_make_maps(const __nv_bfloat16* adig, const __nv_bfloat16* xdig, int64_t n, int64_t ld, CUtensorMap* maps);
// One launch splitting X of every request (its columns, the padding columns to zero), then one launch of the
// residual over all row tiles (first[k]: the first tile of request k, tiles in all); device arrays.
cudaError_t launch_oz_grouped(const OzResidParams* ps_dev, const CUtensorMap* maps_dev, const int64_t* first_dev,
                              int nreq, int64_t tiles, cudaStream_t s);

bool mrhs_supported_r(int64_t r);
// Encodes the TMA maps of the BF16 matrix (n x n, row pitch ld) and of the BF16 iterate block (r x n,
// row pitch ld) and launches one sweep.
cudaError_t launch_mrhs_sweep(const void* Nlow, const void* dh, const MrhsSweepParams& p, cudaStream_t s);
cudaError_t launch_mrhs_dense(const MrhsDenseParams& p, cudaStream_t s);
// xs[c*ld + i] = the two FP32 words of x_ic 2^-g_c, xexp[c] = g_c (the split exponent of max_i |x_ic|).
cudaError_t launch_mrhs_split_x(int64_t n, int64_t r, int64_t ld, const double* x, float2* xs, int* xexp,
                                cudaStream_t s);
// Residual of the zero start vector (R = B): c1 = B / a_ii, d1 = c1 (FP32, BF16), colmax = max |B|.
cudaError_t launch_mrhs_init(int64_t n, int64_t r, int64_t ld, const double* b, const double* rinv, float* c1,
                             float* d1, __nv_bfloat16* d1h, unsigned long long* colmax, cudaStream_t s);

}  // namespace jac
