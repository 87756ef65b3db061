// Shared declarations of the CUDA solver library (kernels <-> host C-ABI layer).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "jacobi.h"

namespace jac {

// ---------------------------------------------------------------- persistent streaming kernels
// Warp layout of the persistent CTA (compile-time; the defaults are the measured best on GB300):
// JAC_COL_WARPS warps split the columns of a ring item, JAC_ROW_GROUPS groups of 8 rows split its rows,
// plus one producer warp.
#ifndef JAC_COL_WARPS
#define JAC_COL_WARPS 7
#endif
#ifndef JAC_ROW_GROUPS
#define JAC_ROW_GROUPS 2
#endif
#ifndef JAC_RING_KB
#define JAC_RING_KB 192
#endif
constexpr int kColWarps = JAC_COL_WARPS;                 // warps across the columns of a ring item
constexpr int kRowsPerWarp = 8;                          // rows each consumer warp accumulates
constexpr int kRowHalves = JAC_ROW_GROUPS;               // warp groups splitting the item's rows
constexpr int kConsumerWarps = kColWarps * kRowHalves;   // warps that compute dot products
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + 32;                // + one producer warp (bulk copies)
// The register file is split over the SM's 4 schedulers (16 K registers each) and a warp lives on
// one of them, so the per-thread budget follows from the warps per scheduler.
constexpr int kWarpsPerScheduler = (kThreads / 32 + 3) / 4;
constexpr int kMaxRegsRaw = 16384 / (kWarpsPerScheduler * 32) / 8 * 8;
constexpr int kMaxRegs = kMaxRegsRaw > 255 ? 255 : kMaxRegsRaw;
constexpr int kRows = kRowsPerWarp * kRowHalves;         // rows of a row group (one ring item)
constexpr int kRowBytes = kColWarps * 32 * 16;           // bytes of one row per ring item
constexpr int kStageBytes = kRows * kRowBytes;           // bytes per ring stage
constexpr int kStages = (JAC_RING_KB * 1024) / kStageBytes;  // ring depth within JAC_RING_KB KB
constexpr int kDynSmem = kStages * kStageBytes + 128;    // + alignment slack
static_assert(kRows <= 32, "one epilogue lane per row of a group");
static_assert(kStages >= 2, "ring needs two stages");
constexpr int kMaxGrid = 1024;                           // size of the per-CTA partial-sum arrays
constexpr int kLdAlign = 16;                             // leading dimensions are multiples of 16

constexpr int kTraceCap = 512;                           // phases recorded by the device-side trace

// Control block of one solve (device memory, zeroed before each launch).
struct Ctl {
  unsigned int arrive;               // grid-barrier arrival counter
  int status;                        // < 0 once any CTA hit an error (timeout)
  unsigned long long red[3][2];      // rotating reduction slots (order-free max of |.| bits)
  jacobi_stats result;               // written by CTA 0 at the end
  // trace: %globaltimer when CTA 0 leaves the grid barrier that ends each phase, and the phase kind
  unsigned long long t_start;
  int nphase;
  int pad_;
  unsigned long long t_end[kTraceCap];
  int kind[kTraceCap];
};

enum class Narrow : int { F32 = 1, BF16 = 2, E4M3 = 3 };

struct SolveParams {
  int64_t n;
  const double* A;        // FP64 A including the diagonal, row-major, row stride lda (16-B aligned rows)
  int64_t lda;
  const void* Nlow;       // IR: narrow off-diagonal copy, row stride ldn, zero diagonal
  int64_t ldn;
  void* Nlow_w;           // the same buffer, written by the first inner sweep when *nready == 0
  int* nready;            // BF16 / FP32 inner sweeps: 0 until the narrow copy and rowfac are written; else NULL
  float* rowfac_w;        // rowfac, written with the narrow copy
  const double* b;        // n
  const double* d;        // n, a_ii
  const double* rinv;     // n, 1 / a_ii (correctly rounded)
  const float* rowfac;    // IR: n, factor of the narrow row dot (1/a_ii, times the E4M3 row scale)
  const double* bnorm;    // ||B||_inf (one value)
  double* xa;             // FP64 iterate buffers, length >= round_up(n, 16), zero padding
  double* xb;
  float2* xsa;            // split-float residual: FP32 (hi, lo) words of xa / xb, else NULL
  float2* xsb;
  float* c1;              // IR: inner right-hand side D^-1 r
  float* da;              // IR: inner iterate buffers
  float* db;
  double* part;           // [2][kMaxGrid] per-CTA partial sums (Euclidean norm)
  Ctl* ctl;
  double* x_out;          // device result (n)
  jacobi_stats* stats_out;  // optional device copy of the result record
  int64_t max_iter;
  double tol;
  int norm;               // jacobi_norm
  int x0_zero;            // 1: the start vector is zero (the first IR residual needs no matrix pass)
  int max_outer;
  int max_inner;
  float inner_rtol;
  const int* rexp;        // IR: per-row scale exponent; non-NULL selects the split-float FP64 residual
  const unsigned long long* cmax;  // split: bits of max_i |b_i / a_ii|, the iterate's scale
  uint64_t wait_ns;       // limit of every device-side wait (nanoseconds)
  int test_drop_copy;     // test only: the first ring item is announced but never copied (a wait expires)
};

// Host launchers (solve.cu).  Each returns a cudaError_t from the launch.
cudaError_t launch_fp64_solve(const SolveParams& p, int grid, cudaStream_t s);
cudaError_t launch_ir_solve(Narrow kind, const SolveParams& p, int grid, cudaStream_t s);
int max_coresident_grid(bool ir, Narrow kind);

// Preparation kernels (prepare.cu).
// Reads a_ii, checks it (zero / non-finite), writes d, rinv; key_out receives the smallest
// (row << 8 | code) of a failing row (code 2: zero, 3: non-finite), or all ones if none.
cudaError_t launch_diag(const double* A, int64_t lda, int64_t n, double* d, double* rinv,
                        unsigned long long* key_out, cudaStream_t s);
// b (FP64 copy), ||b||_inf bits into *bnorm_bits and, unless cmax_bits is NULL, max_i |b_i / a_ii| bits
// into *cmax_bits (both zeroed before; rinv from launch_diag, may be NULL without cmax_bits).
cudaError_t launch_rhs(const double* B, int64_t n, const double* rinv, double* b, unsigned long long* bnorm_bits,
                       unsigned long long* cmax_bits, cudaStream_t s);
// Narrow copy of the off-diagonal part of A (zero diagonal, zero padding up to ldn) and the FP32
// per-row factor of the inner sweep.
// rexp (may be NULL): per row, the exponent e with max_j |a_ij| < 2^e (the split-float residual's scale).
cudaError_t launch_narrow(Narrow kind, const double* A, int64_t lda, int64_t n, void* Nlow, int64_t ldn,
                          const double* rinv, float* scale, float* rowfac, int* rexp, cudaStream_t s);
// xs[i] = the two FP32 words of x_i 2^-g for i < n, g = split_exponent(*cmax_bits): the split-float
// residual's view of a start vector.
cudaError_t launch_split_x(const double* x, int64_t n, const unsigned long long* cmax_bits, float2* xs,
                           cudaStream_t s);
// Zero columns [n, ld) of an n x ld row-major FP64 matrix.
cudaError_t launch_pad_zero(double* M, int64_t n, int64_t ld, cudaStream_t s);
// Relative residual ||b - A x||_inf / ||b||_inf (FP64) into *rel_bits (zeroed before) as max bits of
// |r_i|; the host divides by ||b||.
cudaError_t launch_residual(const double* A, int64_t lda, int64_t n, const double* b, const double* x,
                            unsigned long long* rmax_bits, cudaStream_t s);

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace jac
