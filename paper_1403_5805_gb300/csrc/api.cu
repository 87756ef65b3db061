// C ABI of the solver library (declared in include/jacobi.h): handles, workspace layout, launches.
//
// The problem statement follows Section 2 of the paper: inputs A (alpha_ii != 0), B, the start vector
// X^0, the tolerance and the iteration limit L; output X.  All arithmetic runs in the kernels of
// prepare.cu and solve.cu; this file only validates arguments, lays out device memory and orders the
// work on the handle's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "gs.cuh"
#include "mrhs.cuh"
#include "sym.cuh"
#include "solver.cuh"
#include "sparse.cuh"

using namespace jac;

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return JACOBI_ERR_OUT_OF_MEMORY;
  return JACOBI_ERR_CUDA;
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t narrow_size(int precision) {
  switch (precision) {
    case JACOBI_FP32_IR: return 4;
    case JACOBI_BF16_IR: return 2;
    case JACOBI_FP8_IR: return 1;
    default: return 0;
  }
}

Narrow narrow_kind(int precision) {
  return precision == JACOBI_FP32_IR ? Narrow::F32 : precision == JACOBI_BF16_IR ? Narrow::BF16 : Narrow::E4M3;
}

bool is_device_memory(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown host pointer
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// The sweep streams A in place when its rows are 16-byte aligned device memory (no padding overread:
// n even); host memory and other layouts are copied into the workspace.
bool can_borrow(const jacobi_desc* d) {
  if (!d->A || (d->flags & JACOBI_FLAG_COPY_A)) return false;
  if (reinterpret_cast<uintptr_t>(d->A) % 16 != 0 || d->n % 2 != 0 || d->lda % 2 != 0) return false;
  return is_device_memory(d->A);
}

// Offsets of every sub-buffer inside one workspace allocation.
struct Layout {
  int64_t ld;  // padded length of vectors and row stride of owned matrices
  size_t A64, Nlow, nready, b, d, rinv, bnorm, cmax, rowfac, scale, rexp, xa, xb, xsa, xsb, xout, c1, da, db, part, gsflags,
      gsmbox, ctl, keys, stats, symP, symstats, total;
};

// sym: the narrow copy holds the packed upper tiles of a symmetric A (plus the tile partial sums).
Layout make_layout(int64_t n, int precision, bool copy_A, bool sym = false) {
  Layout L{};
  L.ld = round_up(n, kLdAlign);
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t vd = static_cast<size_t>(L.ld) * sizeof(double);
  const size_t vf = static_cast<size_t>(L.ld) * sizeof(float);
  L.A64 = copy_A ? take(static_cast<size_t>(n) * L.ld * sizeof(double)) : 0;
  const size_t ns = narrow_size(precision);
  if (sym) {
    const int64_t nt = sym_tiles_per_side(n);
    L.Nlow = take(static_cast<size_t>(sym_tile_count(n)) * kSymTile * kSymTile * ns);
    L.symP = take(static_cast<size_t>(nt) * nt * kSymTile * sizeof(float));
    L.symstats = take(4 * sizeof(unsigned long long));
  } else {
    L.Nlow = ns ? take(static_cast<size_t>(n) * L.ld * ns) : 0;
  }
  L.nready = take(sizeof(int));  // nonzero once the narrow copy and rowfac hold this handle's A
  L.b = take(vd);
  L.d = take(vd);
  L.rinv = take(vd);
  L.bnorm = take(sizeof(double));
  L.cmax = take(sizeof(double));
  L.rowfac = take(vf);
  L.scale = take(vf);
  L.rexp = take(static_cast<size_t>(L.ld) * sizeof(int));
  L.xa = take(vd);
  L.xb = take(vd);
  L.xsa = take(2 * vf);  // (hi, lo) FP32 words of xa / xb for the split-float residual
  L.xsb = take(2 * vf);
  L.xout = take(vd);
  L.c1 = take(vf);
  L.da = take(vf);
  L.db = take(vf);
  L.part = take(3 * kMaxGrid * sizeof(double));  // Euclidean-norm partials: 2 slots (Jacobi), 3 (Gauss-Seidel)
  L.gsflags = take(kMaxGrid * sizeof(int));  // Gauss-Seidel chain: per-CTA published sweep
  L.gsmbox = take(2 * vd);                    // Gauss-Seidel chain: mailboxes of x^(k), k odd / even
  L.ctl = take(sizeof(Ctl));
  L.keys = take(4 * sizeof(unsigned long long));
  L.stats = take(sizeof(jacobi_stats));
  L.total = o;
  return L;
}

int validate_desc(const jacobi_desc* d) {
  if (!d || d->n < 1 || d->nrhs < 1 || !d->A || !d->B) return JACOBI_ERR_INVALID_ARG;
  if (d->lda < d->n || d->ldb < d->n) return JACOBI_ERR_INVALID_ARG;
  if (d->precision < JACOBI_FP64 || d->precision > JACOBI_FP8_IR) return JACOBI_ERR_INVALID_ARG;
  if (d->norm < JACOBI_NORM_INF || d->norm > JACOBI_NORM_RESID) return JACOBI_ERR_INVALID_ARG;
  if (d->grid < 0 || d->grid > kMaxGrid) return JACOBI_ERR_INVALID_ARG;
  if (d->method != JACOBI_METHOD_JACOBI && d->method != JACOBI_METHOD_SOR) return JACOBI_ERR_INVALID_ARG;
  if (d->method == JACOBI_METHOD_SOR) {
    if (d->omega != 0.0 && !(d->omega > 0.0 && d->omega < 2.0)) return JACOBI_ERR_INVALID_ARG;
    if (d->precision != JACOBI_FP64 || d->nrhs != 1 || d->norm == JACOBI_NORM_RESID) return JACOBI_ERR_UNSUPPORTED;
  }
  if (d->nrhs > 1) {
    // many right-hand sides: plain FP64 (any stopping norm) or BF16 inner sweeps on tcgen05
    if (d->precision != JACOBI_FP64 && d->precision != JACOBI_BF16_IR) return JACOBI_ERR_UNSUPPORTED;
    if (d->precision == JACOBI_BF16_IR && !mrhs_supported_r(d->nrhs)) return JACOBI_ERR_UNSUPPORTED;
  }
  if (d->flags & JACOBI_FLAG_SYMMETRIC) {
    if (d->flags & (JACOBI_FLAG_SPLIT_RESIDUAL | JACOBI_FLAG_TC_RESIDUAL)) return JACOBI_ERR_INVALID_ARG;
    if (d->nrhs != 1 || d->method != JACOBI_METHOD_JACOBI ||
        (d->precision != JACOBI_BF16_IR && d->precision != JACOBI_FP32_IR))
      return JACOBI_ERR_UNSUPPORTED;
  }
  if (d->flags & JACOBI_FLAG_TC_RESIDUAL) {
    if (d->flags & JACOBI_FLAG_SPLIT_RESIDUAL) return JACOBI_ERR_INVALID_ARG;
    if (d->nrhs < 2 || d->precision != JACOBI_BF16_IR || d->method != JACOBI_METHOD_JACOBI)
      return JACOBI_ERR_UNSUPPORTED;
  }
  return JACOBI_OK;
}

// Extra device buffers of a many-right-hand-side handle (vectors v[c*ld + i]).
struct MrhsLayout {
  size_t b, xa, xb, c1, da, db, dah, dbh, colmax, colsq, bcol, stats, status, xs, xexp, cols, adig, aexp, xdig,
      opart, total;
};

// tc: the tensor-core residual's digit matrices of A (kOzDigits x nr x ld BF16), row exponents, the
// digits of X (kOzDigits x r x ld BF16) and the partial sums of its K-split tiles (kOzMaxParts x r x ld
// float-float).
MrhsLayout mrhs_layout(size_t base, int64_t n, int64_t ld, int64_t r, bool tc) {
  MrhsLayout M{};
  size_t o = base;
  auto take = [&o](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t v8 = static_cast<size_t>(ld) * r * 8, v4 = static_cast<size_t>(ld) * r * 4,
               v2 = static_cast<size_t>(ld) * r * 2;
  M.b = take(v8);
  M.xa = take(v8);
  M.xb = take(v8);
  M.c1 = take(v4);
  M.da = take(v4);
  M.db = take(v4);
  M.dah = take(v2);
  M.dbh = take(v2);
  M.colmax = take(static_cast<size_t>(r) * 8);
  // Euclidean norm: per row tile of the FP64 dense pass and column
  M.colsq = take(static_cast<size_t>((ld + kMrhsDenseRows - 1) / kMrhsDenseRows) * r * 8);
  M.bcol = take(static_cast<size_t>(r) * 8);
  M.stats = take(16);
  M.status = take(16);
  M.xs = take(v8);  // split-float residual: two FP32 words per entry of X
  M.xexp = take(static_cast<size_t>(r) * 4);
  M.cols = take(static_cast<size_t>(r) * 4);  // active columns (column retirement)
  if (tc) {
    const int64_t nr = oz_padded_rows(n);
    M.adig = take(static_cast<size_t>(kOzDigits) * nr * ld * 2);
    M.aexp = take(static_cast<size_t>(nr) * 4);
    M.xdig = take(static_cast<size_t>(kOzDigits) * r * ld * 2);
    M.opart = take(static_cast<size_t>(kOzMaxParts) * r * ld * 8);
  }
  M.total = o;
  return M;
}

}  // namespace

struct jacobi_handle {
  int device = 0;
  int64_t n = 0;
  int64_t nrhs = 1;
  MrhsLayout M{};
  // host-driven paths: per-phase trace from CUDA events (kind, end time since the solve started)
  std::vector<int32_t> htrace_kind;
  std::vector<int64_t> htrace_end;
  int precision = JACOBI_FP64;
  int norm = JACOBI_NORM_INF;
  cudaStream_t stream = nullptr;
  bool own_ws = false;
  char* ws = nullptr;
  Layout L{};
  const double* A64 = nullptr;
  int64_t lda64 = 0;
  int grid = 0;
  int max_outer = 60;
  int max_inner = 1000;
  float inner_rtol = 0.0f;
  bool split_residual = false;
  bool tc_residual = false;  // many right-hand sides: residuals on the tensor cores (digit split of A, X)
  bool symmetric = false;    // symmetric A: packed upper tiles for the narrow inner sweeps (sym.cu)
  bool fuse_narrow = false;  // the narrow copy is written by the first inner sweep of the first solve
  bool retire_columns = false;
  int method = JACOBI_METHOD_JACOBI;
  double omega = 1.0;
  std::vector<int64_t> col_iters;  // per-column record of the last many-right-hand-side solve
  std::vector<double> col_value;
  uint64_t wait_ns = 4000000000ull;
  int test_drop_copy = 0;
  int test_skip_arrival = 0;  // Gauss-Seidel test hook (JACOBI_FLAG_TEST_SKIP_ARRIVAL)
  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
};

namespace {

// The setup pass that writes the narrow copy of A (and rowfac, scale, rexp) and marks it written.
cudaError_t write_narrow(jacobi_handle* h) {
  if (h->symmetric) {
    cudaError_t e = launch_sym_pack(narrow_kind(h->precision), h->A64, h->lda64, h->n, h->at<double>(h->L.rinv),
                                    h->at<void>(h->L.Nlow), h->at<float>(h->L.rowfac), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->at<char>(h->L.nready), 1, sizeof(int), h->stream);
    return e;
  }
  cudaError_t e = launch_narrow(narrow_kind(h->precision), h->A64, h->lda64, h->n, h->at<void>(h->L.Nlow), h->L.ld,
                                h->at<double>(h->L.rinv), h->at<float>(h->L.scale), h->at<float>(h->L.rowfac),
                                h->split_residual ? h->at<int>(h->L.rexp) : nullptr, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->at<char>(h->L.nready), 1, sizeof(int), h->stream);
  return e;
}

// Runs the preparation kernels on h's stream.  A and B are device pointers (or, for the host-pointer
// entry point, A has already been placed in the workspace and B in b).
int prepare(jacobi_handle* h, const double* A, int64_t lda, const double* B, bool copy_A) {
  const int64_t n = h->n;
  cudaStream_t s = h->stream;
  if (copy_A) {
    double* dst = h->at<double>(h->L.A64);
    if (A != dst)
      CK(cudaMemcpy2DAsync(dst, h->L.ld * sizeof(double), A, lda * sizeof(double), n * sizeof(double), n,
                           cudaMemcpyDefault, s));
    CK(launch_pad_zero(dst, n, h->L.ld, s));
    h->A64 = dst;
    h->lda64 = h->L.ld;
  } else {
    h->A64 = A;
    h->lda64 = lda;
  }
  unsigned long long* keys = h->at<unsigned long long>(h->L.keys);
  CK(cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long), s));       // diagonal-check key
  CK(launch_diag(h->A64, h->lda64, n, h->at<double>(h->L.d), h->at<double>(h->L.rinv), keys, s));
  double* b = h->at<double>(h->L.b);
  if (B != b && !is_device_memory(B)) {
    CK(cudaMemcpyAsync(b, B, n * sizeof(double), cudaMemcpyHostToDevice, s));
    B = b;
  }
  // The diagonal decides the return value, so it is checked before the remaining setup work is queued;
  // that work (the narrow copy above all) then runs while the caller goes on to launch the solve.  Every
  // read of caller memory (A and B) is complete at this synchronisation.
  unsigned long long key = 0;
  CK(cudaMemcpyAsync(&key, keys, sizeof(key), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (key != ~0ull) return (key & 0xFF) == 2 ? JACOBI_ERR_ZERO_DIAGONAL : JACOBI_ERR_NONFINITE;
  CK(cudaMemsetAsync(h->at<char>(h->L.bnorm), 0, sizeof(double), s));   // ||B|| bits
  CK(cudaMemsetAsync(h->at<char>(h->L.cmax), 0, sizeof(double), s));    // max |b_i / a_ii| bits
  CK(launch_rhs(B, n, h->at<double>(h->L.rinv), b, h->at<unsigned long long>(h->L.bnorm),
                h->at<unsigned long long>(h->L.cmax), s));
  // vectors start zeroed so that every padding entry is 0
  CK(cudaMemsetAsync(h->at<char>(h->L.xa), 0, h->L.ld * sizeof(double), s));
  CK(cudaMemsetAsync(h->at<char>(h->L.xb), 0, h->L.ld * sizeof(double), s));
  CK(cudaMemsetAsync(h->at<char>(h->L.xsa), 0, h->L.ld * sizeof(float2), s));
  CK(cudaMemsetAsync(h->at<char>(h->L.xsb), 0, h->L.ld * sizeof(float2), s));
  CK(cudaMemsetAsync(h->at<char>(h->L.c1), 0, h->L.ld * sizeof(float), s));
  CK(cudaMemsetAsync(h->at<char>(h->L.da), 0, h->L.ld * sizeof(float), s));
  CK(cudaMemsetAsync(h->at<char>(h->L.db), 0, h->L.ld * sizeof(float), s));
  CK(cudaMemsetAsync(h->at<char>(h->L.nready), 0, sizeof(int), s));
  if (h->precision != JACOBI_FP64 && !h->fuse_narrow) CK(write_narrow(h));
  if (h->method == JACOBI_METHOD_SOR) CK(launch_gs_row_exponents(h->A64, h->lda64, n, h->at<int>(h->L.rexp), s));
  return JACOBI_OK;
}

int pick_grid(jacobi_handle* h, int requested) {
  const bool ir = h->precision != JACOBI_FP64;
  const int cap = max_coresident_grid(ir, narrow_kind(h->precision));
  if (cap <= 0) return 0;
  int g = requested > 0 ? requested : static_cast<int>((h->n + kRows - 1) / kRows);
  if (g > cap) g = cap;
  if (g > kMaxGrid) g = kMaxGrid;
  if (g < 1) g = 1;
  return g;
}

// Grid of the chained Gauss-Seidel kernel: by default the fewest row blocks of at most kGsMaxRows rows
// (a requested grid is honoured within that bound); -1 if n needs more blocks than can be co-resident,
// 0 on a failed query.
int pick_gs_grid(int64_t n, int requested) {
  const int cap = gs_max_grid();
  if (cap <= 0) return 0;
  const int64_t need = (n + kGsMaxRows - 1) / kGsMaxRows;
  if (need > cap || need > kMaxGrid) return -1;
  // default: the fewest, largest row blocks (the chain's hand-offs cost more than the block products)
  int64_t g = requested > 0 ? requested : need;
  g = std::min<int64_t>({g, static_cast<int64_t>(cap), static_cast<int64_t>(kMaxGrid), n});
  return static_cast<int>(std::max<int64_t>(g, need));
}

int make_handle(const jacobi_desc* d, bool copy_A, jacobi_handle** out) {
  jacobi_handle* h = new (std::nothrow) jacobi_handle();
  if (!h) return JACOBI_ERR_OUT_OF_MEMORY;
  cudaGetDevice(&h->device);
  h->n = d->n;
  h->precision = d->precision;
  h->norm = d->norm;
  h->stream = static_cast<cudaStream_t>(d->stream);
  h->symmetric = (d->flags & JACOBI_FLAG_SYMMETRIC) != 0;
  h->L = make_layout(d->n, d->precision, copy_A, h->symmetric);
  h->nrhs = d->nrhs;
  if (h->nrhs > 1) {
    h->tc_residual = (d->flags & JACOBI_FLAG_TC_RESIDUAL) != 0;
    h->M = mrhs_layout(h->L.total, h->n, h->L.ld, h->nrhs, h->tc_residual);
    h->L.total = h->M.total;
  }
  h->max_outer = d->max_outer > 0 ? d->max_outer : 60;
  h->max_inner = d->max_inner > 0 ? d->max_inner : 1000;
  h->inner_rtol = static_cast<float>(
      d->inner_rtol > 0 ? d->inner_rtol : (d->precision == JACOBI_FP8_IR ? 1.0 / 64 : 1.0 / 1024));
  h->split_residual = (d->flags & JACOBI_FLAG_SPLIT_RESIDUAL) && d->precision != JACOBI_FP64;
  h->retire_columns = (d->flags & JACOBI_FLAG_RETIRE_COLUMNS) && d->nrhs > 1;
  // BF16 / FP32 copies need no row scale, so a single-right-hand-side solve can round A while it streams
  // it for its first inner sweep instead of a separate setup pass over A
  h->fuse_narrow = d->nrhs == 1 && d->method == JACOBI_METHOD_JACOBI && !h->split_residual && !h->symmetric &&
                   (d->precision == JACOBI_BF16_IR || d->precision == JACOBI_FP32_IR);
  if (d->flags & JACOBI_FLAG_SHORT_WAITS) h->wait_ns = 50000000ull;
  h->test_drop_copy = (d->flags & JACOBI_FLAG_TEST_DROP_COPY) ? 1 : 0;
  h->test_skip_arrival = (d->flags & JACOBI_FLAG_TEST_SKIP_ARRIVAL) ? 1 : 0;
  if (d->workspace) {
    if (d->workspace_bytes < h->L.total || reinterpret_cast<uintptr_t>(d->workspace) % kAlign != 0) {
      delete h;
      return JACOBI_ERR_INVALID_ARG;
    }
    h->ws = static_cast<char*>(d->workspace);
  } else {
    cudaError_t e = cudaMalloc(&h->ws, h->L.total);
    if (e != cudaSuccess) {
      delete h;
      return cuda_fail(e, "cudaMalloc(workspace)");
    }
    h->own_ws = true;
  }
  h->method = d->method;
  h->omega = d->omega > 0.0 ? d->omega : 1.0;
  h->grid = h->method == JACOBI_METHOD_SOR ? pick_gs_grid(h->n, d->grid) : pick_grid(h, d->grid);
  if (h->grid == -1) {
    if (h->own_ws) cudaFree(h->ws);
    delete h;
    return JACOBI_ERR_UNSUPPORTED;  // n too large for the chained Gauss-Seidel blocks
  }
  if (h->grid <= 0) {
    if (h->own_ws) cudaFree(h->ws);
    delete h;
    return cuda_fail(cudaGetLastError(), "occupancy query");
  }
  *out = h;
  return JACOBI_OK;
}

// B (column-major, ldb) into the padded column layout and ||b_c||_inf per column.
int mrhs_prepare(jacobi_handle* h, const double* B, int64_t ldb) {
  cudaStream_t s = h->stream;
  const int64_t n = h->n, r = h->nrhs, ld = h->L.ld;
  double* b = h->at<double>(h->M.b);
  CK(cudaMemsetAsync(b, 0, static_cast<size_t>(ld) * r * 8, s));
  CK(cudaMemcpy2DAsync(b, ld * sizeof(double), B, ldb * sizeof(double), n * sizeof(double), r, cudaMemcpyDefault, s));
  for (size_t off : {h->M.xa, h->M.xb})
    CK(cudaMemsetAsync(h->at<char>(off), 0, static_cast<size_t>(ld) * r * 8, s));
  for (size_t off : {h->M.c1, h->M.da, h->M.db})
    CK(cudaMemsetAsync(h->at<char>(off), 0, static_cast<size_t>(ld) * r * 4, s));
  for (size_t off : {h->M.dah, h->M.dbh})
    CK(cudaMemsetAsync(h->at<char>(off), 0, static_cast<size_t>(ld) * r * 2, s));
  // per-column ||b||: the init kernel's column maxima of |B|
  unsigned long long* bcol = h->at<unsigned long long>(h->M.bcol);
  CK(cudaMemsetAsync(bcol, 0, static_cast<size_t>(r) * 8, s));
  CK(launch_mrhs_init(n, r, ld, b, h->at<double>(h->L.rinv), h->at<float>(h->M.c1), h->at<float>(h->M.da),
                      h->at<__nv_bfloat16>(h->M.dah), bcol, s));
  if (h->tc_residual)
    CK(launch_oz_split_a(h->A64, h->lda64, n, ld, h->at<__nv_bfloat16>(h->M.adig), h->at<int>(h->M.aexp), s));
  CK(cudaStreamSynchronize(s));
  return JACOBI_OK;
}

// Host-driven loop for many right-hand sides (each FP64 pass over A is a full matrix-matrix product,
// milliseconds to a hundred milliseconds, so one small device-to-host read per phase costs nothing).
// CUDA-event timeline of a host-driven solve: one event after every phase.
struct PhaseClock {
  cudaStream_t s;
  std::vector<cudaEvent_t> ev;
  std::vector<int32_t> kind;
  explicit PhaseClock(cudaStream_t st) : s(st) { mark(-1); }
  void mark(int32_t k) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s);
    ev.push_back(e);
    kind.push_back(k);
  }
  // after a stream synchronisation: fill the handle's trace
  void flush(jacobi_handle* h) {
    h->htrace_kind.clear();
    h->htrace_end.clear();
    for (size_t i = 1; i < ev.size(); ++i) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev[0], ev[i]);
      h->htrace_kind.push_back(kind[i]);
      h->htrace_end.push_back(static_cast<int64_t>(static_cast<double>(ms) * 1e6));
    }
  }
  ~PhaseClock() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

int mrhs_solve(jacobi_handle* h, const double* X0, int64_t max_iter, double tol, double* X_out, jacobi_stats* st) {
  cudaStream_t s = h->stream;
  PhaseClock clk(s);
  const int64_t n = h->n, r = h->nrhs, ld = h->L.ld;
  double* xa = h->at<double>(h->M.xa);
  double* xb = h->at<double>(h->M.xb);
  unsigned long long* colmax = h->at<unsigned long long>(h->M.colmax);
  int* dcols = h->at<int>(h->M.cols);
  std::vector<unsigned long long> hc(static_cast<size_t>(r)), hb(static_cast<size_t>(r));
  CK(cudaMemcpyAsync(hb.data(), h->at<char>(h->M.bcol), static_cast<size_t>(r) * 8, cudaMemcpyDeviceToHost, s));
  if (X0)
    CK(cudaMemcpy2DAsync(xa, ld * 8, X0, n * 8, n * 8, r, cudaMemcpyDefault, s));
  else
    CK(cudaMemsetAsync(xa, 0, static_cast<size_t>(ld) * r * 8, s));
  auto bits = [](unsigned long long u) {
    double v;
    std::memcpy(&v, &u, 8);
    return v;
  };
  // Active columns (all of them unless retirement is on); a retired column's final iterate goes to X_out
  // when it retires, the others' at the end.
  const bool retire = h->retire_columns;
  std::vector<int> act(static_cast<size_t>(r));
  for (int64_t c = 0; c < r; ++c) act[static_cast<size_t>(c)] = static_cast<int>(c);
  h->col_iters.assign(static_cast<size_t>(r), 0);
  h->col_value.assign(static_cast<size_t>(r), std::nan(""));
  auto copy_out = [&](int c, const double* x) -> cudaError_t {
    return cudaMemcpyAsync(X_out + static_cast<int64_t>(c) * n, x + static_cast<int64_t>(c) * ld, n * 8,
                           cudaMemcpyDefault, s);
  };
  auto upload_active = [&]() -> cudaError_t {
    return cudaMemcpyAsync(dcols, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  };
  jacobi_stats out{};
  out.rel_residual = std::nan("");
  out.status = JACOBI_NOT_CONVERGED;
  double* xc = xa;
  double* xo = xb;
  bool all_retired = false;
  if (h->precision == JACOBI_FP64) {
    const int resid = h->norm == JACOBI_NORM_RESID;
    const bool eucl = h->norm == JACOBI_NORM_2;
    const int64_t tiles = (n + kMrhsDenseRows - 1) / kMrhsDenseRows;
    double* colsq = h->at<double>(h->M.colsq);
    std::vector<double> hs(eucl ? static_cast<size_t>(tiles * r) : 0);
    for (int64_t k = 1;; ++k) {
      CK(cudaMemsetAsync(colmax, 0, static_cast<size_t>(r) * 8, s));
      if (retire) CK(upload_active());
      MrhsDenseParams p{n, r, ld, h->lda64, 1, resid, h->A64, h->at<double>(h->M.b), xc, h->at<double>(h->L.d),
                        h->at<double>(h->L.rinv), nullptr, nullptr, nullptr, xo, colmax, nullptr, nullptr, nullptr,
                        retire ? dcols : nullptr, static_cast<int64_t>(act.size()), eucl ? colsq : nullptr};
      CK(launch_mrhs_dense(p, s));
      clk.mark(JACOBI_PHASE_SWEEP64);
      CK(cudaMemcpyAsync(hc.data(), colmax, static_cast<size_t>(r) * 8, cudaMemcpyDeviceToHost, s));
      if (eucl) CK(cudaMemcpyAsync(hs.data(), colsq, hs.size() * 8, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      std::swap(xc, xo);  // xc: the iterate this sweep produced
      double delta = 0.0;
      std::vector<int> keep;
      for (int c : act) {
        // max-norm change of the column, its Euclidean norm (the tiles' sums added in tile order, Section
        // 2's criterion), or its relative residual of the previous iterate
        // (max_i |a_ii (x_i^(k) - x_i^(k-1))| / ||b_c||_inf)
        double v;
        if (eucl) {
          double t = 0.0;
          for (int64_t q = 0; q < tiles; ++q) t += hs[static_cast<size_t>(q * r + c)];
          v = std::sqrt(t);
        } else {
          v = resid ? bits(hc[static_cast<size_t>(c)]) / bits(hb[static_cast<size_t>(c)]) : bits(hc[static_cast<size_t>(c)]);
        }
        delta = (std::isnan(v) || v > delta) ? v : delta;
        h->col_iters[static_cast<size_t>(c)] = k;
        h->col_value[static_cast<size_t>(c)] = v;
        if (retire && v < tol)
          CK(copy_out(c, xc));
        else
          keep.push_back(c);
      }
      out.sweeps = k;
      out.final_delta = delta;
      if (!std::isfinite(delta)) {
        out.status = JACOBI_ERR_NONFINITE;
        break;
      }
      if (retire) {
        act.swap(keep);
        if (act.empty()) {
          out.status = JACOBI_OK;
          all_retired = true;
          break;
        }
      } else if (delta < tol) {
        out.status = JACOBI_OK;
        break;
      }
      if (k >= max_iter) break;
    }
  } else {
    float* c1 = h->at<float>(h->M.c1);
    float* dA = h->at<float>(h->M.da);
    float* dB = h->at<float>(h->M.db);
    __nv_bfloat16* hA = h->at<__nv_bfloat16>(h->M.dah);
    __nv_bfloat16* hB = h->at<__nv_bfloat16>(h->M.dbh);
    unsigned long long* sst = h->at<unsigned long long>(h->M.stats);
    int* status = h->at<int>(h->M.status);
    CK(cudaMemsetAsync(status, 0, sizeof(int), s));
    bool first = (X0 == nullptr);
    int64_t outer = 0, inner_total = 0;
    for (;;) {
      CK(cudaMemsetAsync(colmax, 0, static_cast<size_t>(r) * 8, s));
      if (first) {
        CK(launch_mrhs_init(n, r, ld, h->at<double>(h->M.b), h->at<double>(h->L.rinv), c1, dA, hA, colmax, s));
        clk.mark(JACOBI_PHASE_RESID0);
      } else {
        if (retire) CK(upload_active());
        MrhsDenseParams p{n, r, ld, h->lda64, 0, 0, h->A64, h->at<double>(h->M.b), xc, h->at<double>(h->L.d),
                          h->at<double>(h->L.rinv), c1, dA, hA, nullptr, colmax, nullptr, nullptr, nullptr,
                          retire ? dcols : nullptr, static_cast<int64_t>(act.size())};
        if (h->split_residual) {
          p.rexp = h->at<int>(h->L.rexp);
          p.xs = h->at<float2>(h->M.xs);
          p.xexp = h->at<int>(h->M.xexp);
          CK(launch_mrhs_split_x(n, r, ld, xc, h->at<float2>(h->M.xs), h->at<int>(h->M.xexp), s));
        }
        if (h->tc_residual) {
          OzResidParams q{};
          q.n = n;
          q.r = r;
          q.ld = ld;
          q.nr = oz_padded_rows(n);
          q.aexp = h->at<int>(h->M.aexp);
          q.xexp = h->at<int>(h->M.xexp);
          q.x = xc;
          q.b = h->at<double>(h->M.b);
          q.d = h->at<double>(h->L.d);
          q.rinv = h->at<double>(h->L.rinv);
          q.c1 = c1;
          q.d1 = dA;
          q.d1h = hA;
          q.colmax = colmax;
          q.cols = retire ? dcols : nullptr;
          q.nact = static_cast<int64_t>(act.size());
          q.status = status;
          q.wait_ns = h->wait_ns;
          q.part = h->at<float2>(h->M.opart);
          CK(launch_oz_split_x(n, r, ld, xc, h->at<__nv_bfloat16>(h->M.xdig), h->at<int>(h->M.xexp), s));
          CK(launch_oz_resid(h->at<__nv_bfloat16>(h->M.adig), h->at<__nv_bfloat16>(h->M.xdig), q, s));
        } else {
          CK(launch_mrhs_dense(p, s));
        }
        clk.mark(JACOBI_PHASE_RESID64);
      }
      first = false;
      ++outer;
      CK(cudaMemcpyAsync(hc.data(), colmax, static_cast<size_t>(r) * 8, cudaMemcpyDeviceToHost, s));
      int rst = 0;
      if (h->tc_residual) CK(cudaMemcpyAsync(&rst, status, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (rst != 0) {  // a bounded wait of the tensor-core residual expired: its maxima are incomplete
        out.status = rst;
        break;
      }
      double rho = 0.0;
      std::vector<int> keep;
      for (int c : act) {
        const double v = bits(hc[static_cast<size_t>(c)]) / bits(hb[static_cast<size_t>(c)]);
        rho = (std::isnan(v) || v > rho) ? v : rho;
        h->col_iters[static_cast<size_t>(c)] = outer;
        h->col_value[static_cast<size_t>(c)] = v;
        if (retire && v <= tol) {
          // the residual just measured is that of xc: it is this column's result; its inner
          // right-hand side and iterates are zeroed so the shared inner sweeps carry it at delta = 0
          CK(copy_out(c, xc));
          CK(cudaMemsetAsync(c1 + static_cast<int64_t>(c) * ld, 0, ld * sizeof(float), s));
          CK(cudaMemsetAsync(dA + static_cast<int64_t>(c) * ld, 0, ld * sizeof(float), s));
          CK(cudaMemsetAsync(hA + static_cast<int64_t>(c) * ld, 0, ld * sizeof(__nv_bfloat16), s));
        } else {
          keep.push_back(c);
        }
      }
      out.rel_residual = rho;
      if (!std::isfinite(rho)) {
        out.status = JACOBI_ERR_NONFINITE;
        break;
      }
      if (retire) {
        act.swap(keep);
        if (act.empty()) {
          out.status = JACOBI_OK;
          all_retired = true;
          break;
        }
      } else if (rho <= tol) {
        out.status = JACOBI_OK;
        break;
      }
      if (outer >= h->max_outer || inner_total >= max_iter) break;
      float* dcur = dA;
      float* dnew = dB;
      __nv_bfloat16* hcur = hA;
      __nv_bfloat16* hnew = hB;
      for (int64_t m = 1;; ++m) {
        CK(cudaMemsetAsync(sst, 0, 16, s));
        MrhsSweepParams q{n, r, ld, h->at<float>(h->L.rowfac), c1, dcur, dnew, hnew, xc, xo, sst, status};
        CK(launch_mrhs_sweep(h->at<void>(h->L.Nlow), hcur, q, s));
        clk.mark(JACOBI_PHASE_INNER);
        unsigned long long hs[2];
        int hst = 0;
        CK(cudaMemcpyAsync(hs, sst, 16, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        ++inner_total;
        if (hst != 0) {
          out.status = hst;
          break;
        }
        const double chg = bits(hs[0]), mag = bits(hs[1]);
        out.final_delta = chg;
        std::swap(dcur, dnew);
        std::swap(hcur, hnew);
        if (!std::isfinite(chg) || !std::isfinite(mag)) {
          out.status = JACOBI_ERR_NONFINITE;
          break;
        }
        if (chg <= h->inner_rtol * mag || m >= h->max_inner || inner_total >= max_iter) break;
      }
      if (out.status != JACOBI_NOT_CONVERGED) break;
      std::swap(xc, xo);  // X + delta becomes the current iterate (the next residual rewrites dA / hA)
    }
    out.sweeps = inner_total;
    out.outer_steps = outer;
  }
  if (retire) {
    if (!all_retired)
      for (int c : act) CK(copy_out(c, xc));
  } else {
    CK(cudaMemcpy2DAsync(X_out, n * 8, xc, ld * 8, n * 8, r, cudaMemcpyDefault, s));
  }
  CK(cudaStreamSynchronize(s));
  clk.flush(h);
  out.converged = out.status == JACOBI_OK;
  if (st) *st = out;
  // keep the record where jacobi_last_stats finds it
  CK(cudaMemcpyAsync(&h->at<Ctl>(h->L.ctl)->result, &out, sizeof(out), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return out.status;
}

// Host-driven refinement for a symmetric A (packed upper tiles for the inner sweeps): the control flow of
// the single-system mixed-precision kernel (FP64 residual, inner sweeps until the relative change is at
// most inner_rtol, X + delta, stop at ||B - A X|| / ||B|| <= tol), with one small device-to-host read per
// phase.  The result record goes where jacobi_last_stats finds it; X_out is device or host memory.
int sym_solve(jacobi_handle* h, const double* X0, int64_t max_iter, double tol, double* X_out,
              jacobi_stats* stats_dev) {
  cudaStream_t s = h->stream;
  PhaseClock clk(s);
  const int64_t n = h->n;
  double* xc = h->at<double>(h->L.xa);
  double* xo = h->at<double>(h->L.xb);
  float* c1 = h->at<float>(h->L.c1);
  float* dcur = h->at<float>(h->L.da);
  float* dnew = h->at<float>(h->L.db);
  unsigned long long* st = h->at<unsigned long long>(h->L.symstats);
  if (X0)
    CK(cudaMemcpyAsync(xc, X0, n * sizeof(double), cudaMemcpyDefault, s));
  else
    CK(cudaMemsetAsync(xc, 0, n * sizeof(double), s));
  double bn = 0.0;
  CK(cudaMemcpyAsync(&bn, h->at<double>(h->L.bnorm), sizeof(bn), cudaMemcpyDeviceToHost, s));
  auto bits = [](unsigned long long u) {
    double v;
    std::memcpy(&v, &u, 8);
    return v;
  };
  jacobi_stats out{};
  out.rel_residual = std::nan("");
  out.status = JACOBI_NOT_CONVERGED;
  int64_t outer = 0, inner_total = 0;
  bool first = true;
  for (;;) {
    clk.mark(JACOBI_PHASE_HOST_GAP);  // the phase's own time starts here, after the host's decision
    CK(cudaMemsetAsync(st, 0, 2 * sizeof(unsigned long long), s));
    CK(launch_sym_resid(n, h->A64, h->lda64, (first && !X0) ? nullptr : xc, h->at<double>(h->L.b),
                        h->at<double>(h->L.rinv), c1, h->at<float>(h->L.da), st, s));
    clk.mark((first && !X0) ? JACOBI_PHASE_RESID0 : JACOBI_PHASE_RESID64);
    first = false;
    unsigned long long hs[2];
    CK(cudaMemcpyAsync(hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ++outer;
    const double rho = bits(hs[0]) / bn;
    out.rel_residual = rho;
    if (!std::isfinite(rho)) {
      out.status = JACOBI_ERR_NONFINITE;
      break;
    }
    if (rho <= tol) {
      out.status = JACOBI_OK;
      break;
    }
    if (outer >= h->max_outer || inner_total >= max_iter) break;
    dcur = h->at<float>(h->L.da);  // the residual wrote delta^(1) = c1 there
    dnew = h->at<float>(h->L.db);
    for (int64_t m = 1;; ++m) {
      clk.mark(JACOBI_PHASE_HOST_GAP);
      CK(cudaMemsetAsync(st, 0, 2 * sizeof(unsigned long long), s));
      CK(launch_sym_sweep(narrow_kind(h->precision), h->at<void>(h->L.Nlow), n, dcur, h->at<float>(h->L.symP), c1,
                          h->at<float>(h->L.rowfac), dnew, xc, xo, st, s));
      clk.mark(JACOBI_PHASE_INNER);
      CK(cudaMemcpyAsync(hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      ++inner_total;
      const double chg = bits(hs[0]), mag = bits(hs[1]);
      out.final_delta = chg;
      std::swap(dcur, dnew);
      if (!std::isfinite(chg) || !std::isfinite(mag)) {
        out.status = JACOBI_ERR_NONFINITE;
        break;
      }
      if (chg <= h->inner_rtol * mag || m >= h->max_inner || inner_total >= max_iter) break;
    }
    if (out.status != JACOBI_NOT_CONVERGED) break;
    std::swap(xc, xo);  // X + delta becomes the current iterate
  }
  out.sweeps = inner_total;
  out.outer_steps = outer;
  out.converged = out.status == JACOBI_OK;
  CK(cudaMemcpyAsync(X_out, xc, n * sizeof(double), cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(&h->at<Ctl>(h->L.ctl)->result, &out, sizeof(out), cudaMemcpyHostToDevice, s));
  if (stats_dev) CK(cudaMemcpyAsync(stats_dev, &out, sizeof(out), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  clk.flush(h);
  return JACOBI_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------ sparse A

struct jacobi_csr {
  int device = 0;
  int64_t n = 0, nslices = 0, stored = 0;
  int norm = JACOBI_NORM_INF;
  int grid = 0;
  uint64_t wait_ns = 4000000000ull;
  int test_skip_arrival = 0;
  cudaStream_t stream = nullptr;
  void* mem = nullptr;  // one allocation for everything below
  int64_t* soff = nullptr;
  double* sval = nullptr;
  int32_t* scol = nullptr;
  double* c = nullptr;  // C = D^-1 B
  double* xa = nullptr;
  double* xb = nullptr;
  double* xout = nullptr;
  double* part = nullptr;
  Ctl* ctl = nullptr;
  // mixed precision
  int precision = JACOBI_FP64;
  int max_outer = 60, max_inner = 1000;
  float inner_rtol = 0.0f;
  double bnorm = 0.0;
  void* tlo = nullptr;
  double* d = nullptr;
  float* rf = nullptr;
  float* da = nullptr;
  float* db = nullptr;
  // DIA copy (ndiag > 0): ascending offsets j - i, and the zero halo around the gathered vectors
  int ndiag = 0;
  int32_t* doff = nullptr;
  int64_t halo = 0;
};

namespace {

// Device copies of caller arrays that live on the host (device arrays are used in place); freed on exit.
struct Staged {
  std::vector<void*> owned;
  ~Staged() {
    for (void* p : owned) cudaFree(p);
  }
  template <class T>
  cudaError_t get(const T* src, size_t count, cudaStream_t s, const T** out) {
    if (is_device_memory(src)) {
      *out = src;
      return cudaSuccess;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T) + 16);
    if (e != cudaSuccess) return e;
    owned.push_back(p);
    e = cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyDefault, s);
    *out = static_cast<const T*>(p);
    return e;
  }
};

int csr_setup(const jacobi_csr_desc* d, jacobi_csr** out) {
  if (!d || !out || d->n < 1 || d->nnz < 1 || !d->row_ptr || !d->col_idx || !d->values || !d->B)
    return JACOBI_ERR_INVALID_ARG;
  if (d->norm != JACOBI_NORM_INF && d->norm != JACOBI_NORM_2 && d->norm != JACOBI_NORM_RESID)
    return JACOBI_ERR_INVALID_ARG;
  if (d->n > (int64_t(1) << 31) - 64) return JACOBI_ERR_INVALID_ARG;  // int32 column indices
  if (d->precision < JACOBI_FP64 || d->precision > JACOBI_FP8_IR || d->max_outer < 0 || d->max_inner < 0 ||
      !(d->inner_rtol >= 0.0) || d->inner_rtol >= 1.0)
    return JACOBI_ERR_INVALID_ARG;
  if (d->precision == JACOBI_FP8_IR) return JACOBI_ERR_UNSUPPORTED;
  if (d->precision != JACOBI_FP64 && d->norm != JACOBI_NORM_INF) return JACOBI_ERR_INVALID_ARG;
  *out = nullptr;
  const int64_t n = d->n, nnz = d->nnz;
  cudaStream_t s = static_cast<cudaStream_t>(d->stream);
  int64_t ends[2] = {0, 0};
  CK(cudaMemcpyAsync(&ends[0], d->row_ptr, sizeof(int64_t), cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(&ends[1], d->row_ptr + n, sizeof(int64_t), cudaMemcpyDefault, s));
  CK(cudaStreamSynchronize(s));
  if (ends[0] != 0 || ends[1] != nnz) return JACOBI_ERR_INVALID_ARG;

  Staged st;
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* va = nullptr;
  CK(st.get(d->row_ptr, static_cast<size_t>(n + 1), s, &rp));
  CK(st.get(d->col_idx, static_cast<size_t>(nnz), s, &ci));
  CK(st.get(d->values, static_cast<size_t>(nnz), s, &va));
  const int64_t nslices = (n + kSliceRows - 1) / kSliceRows, npad = nslices * kSliceRows;
  // setup scratch: d (n), lens (npad), widths (nslices), key
  void* scratch = nullptr;
  const size_t sc_bytes = align_up(n * sizeof(double)) + align_up(npad * sizeof(int32_t)) +
                          align_up(nslices * sizeof(int32_t)) + align_up(sizeof(unsigned long long));
  CK(cudaMalloc(&scratch, sc_bytes));
  st.owned.push_back(scratch);
  char* sp = static_cast<char*>(scratch);
  double* dd = reinterpret_cast<double*>(sp);
  int32_t* lens = reinterpret_cast<int32_t*>(sp + align_up(n * sizeof(double)));
  int32_t* width = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(lens) + align_up(npad * sizeof(int32_t)));
  unsigned long long* key =
      reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(width) + align_up(nslices * sizeof(int32_t)));

  std::unique_ptr<jacobi_csr> h(new (std::nothrow) jacobi_csr());
  if (!h) return JACOBI_ERR_OUT_OF_MEMORY;
  cudaGetDevice(&h->device);
  h->n = n;
  h->nslices = nslices;
  h->norm = d->norm;
  h->stream = s;
  if (d->flags & JACOBI_FLAG_SHORT_WAITS) h->wait_ns = 50000000ull;
  h->test_skip_arrival = (d->flags & JACOBI_FLAG_TEST_SKIP_ARRIVAL) ? 1 : 0;
  h->precision = d->precision;
  const bool ir = d->precision != JACOBI_FP64;
  const bool keep_d = ir || d->norm == JACOBI_NORM_RESID;  // a_ii for the residual norm
  if (d->max_outer > 0) h->max_outer = d->max_outer;
  if (d->max_inner > 0) h->max_inner = d->max_inner;
  h->inner_rtol = d->inner_rtol > 0.0 ? static_cast<float>(d->inner_rtol)
                                      : (d->precision == JACOBI_BF16_IR ? 0x1p-8f : 0x1p-20f);

  const size_t vec = align_up(npad * sizeof(double));
  const size_t vecf = align_up(npad * sizeof(float));
  const size_t head = align_up((nslices + 1) * sizeof(int64_t)) + 4 * vec + align_up(2 * kMaxGrid * sizeof(double)) +
                      align_up(sizeof(Ctl)) + align_up(sizeof(unsigned long long)) + (keep_d ? vec : 0) +
                      (ir ? 3 * vecf : 0);
  CK(cudaMemsetAsync(lens, 0, npad * sizeof(int32_t), s));
  CK(cudaMemsetAsync(key, 0xFF, sizeof(unsigned long long), s));
  CK(launch_csr_check(n, nnz, rp, ci, va, dd, lens, key, s));
  unsigned long long hkey = 0;
  CK(cudaMemcpyAsync(&hkey, key, sizeof(hkey), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hkey != ~0ull) {
    if ((hkey >> 56) == 0) return JACOBI_ERR_INVALID_ARG;
    return (hkey & 0xFF) == 3 ? JACOBI_ERR_NONFINITE : JACOBI_ERR_ZERO_DIAGONAL;
  }
  CK(launch_csr_widths(n, lens, width, s));
  std::vector<int32_t> hw(static_cast<size_t>(nslices));
  CK(cudaMemcpyAsync(hw.data(), width, nslices * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<int64_t> hoff(static_cast<size_t>(nslices + 1), 0);
  for (int64_t q = 0; q < nslices; ++q) hoff[q + 1] = hoff[q] + int64_t(kSliceRows) * hw[q];
  const int64_t ell_slots = hoff[nslices];
  // A banded or stencil matrix, whose entries lie on a few diagonals j - i = const, is kept in DIA form:
  // no column array, and contiguous gathers.  The candidate offsets come from a sample of rows; a pass
  // over all entries then confirms that no entry lies off them, and the band must not store many more
  // slots than sliced ELL would.
  std::vector<int32_t> offs;
  if (!(d->flags & JACOBI_FLAG_CSR_ELL)) {
    std::vector<int64_t> rows = {0, n / 4, n / 3, n / 2, 2 * n / 3, 3 * n / 4, n - 1};
    bool ok = true;
    for (int64_t r : rows) {
      int64_t be[2];
      CK(cudaMemcpyAsync(be, rp + r, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (be[1] - be[0] > 2 * kMaxDiag + 1) {
        ok = false;
        break;
      }
      std::vector<int32_t> cols(static_cast<size_t>(be[1] - be[0]));
      if (!cols.empty()) CK(cudaMemcpyAsync(cols.data(), ci + be[0], cols.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int32_t c : cols)
        if (c != r && std::find(offs.begin(), offs.end(), static_cast<int32_t>(c - r)) == offs.end())
          offs.push_back(static_cast<int32_t>(c - r));
    }
    std::sort(offs.begin(), offs.end());
    if (!ok || offs.empty() || offs.size() > static_cast<size_t>(kMaxDiag) ||
        static_cast<double>(offs.size()) * static_cast<double>(npad) > 1.25 * static_cast<double>(ell_slots))
      offs.clear();
    if (!offs.empty()) {  // every entry on a sampled diagonal?  (scratch: the lens array, no longer needed)
      int32_t* doff_s = lens;
      int* bad = reinterpret_cast<int*>(lens + kMaxDiag);
      CK(cudaMemcpyAsync(doff_s, offs.data(), offs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
      CK(launch_csr_dia_check(n, rp, ci, doff_s, static_cast<int>(offs.size()), bad, s));
      int hbad = 0;
      CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (hbad) offs.clear();
    }
  }
  const bool dia = !offs.empty();
  h->ndiag = static_cast<int>(offs.size());
  if (dia) {
    int64_t m = 0;
    for (int32_t o : offs) m = std::max<int64_t>(m, o < 0 ? -static_cast<int64_t>(o) : o);
    h->halo = (m + 31) / 32 * 32;
  }
  const int64_t stored = dia ? static_cast<int64_t>(offs.size()) * npad : ell_slots;
  h->stored = stored;
  const size_t vbytes = align_up(std::max<int64_t>(stored, 1) * sizeof(double));
  const size_t cbytes = dia ? align_up(kMaxDiag * sizeof(int32_t)) : align_up(std::max<int64_t>(stored, 1) * sizeof(int32_t));
  const size_t tbytes = ir ? align_up(std::max<int64_t>(stored, 1) * (d->precision == JACOBI_BF16_IR ? 2 : 4)) : 0;
  // the gathered vectors (x, and the refinement's r' and delta) with their halo on both sides
  const size_t vech = align_up((npad + 2 * h->halo) * sizeof(double));
  const size_t vecfh = align_up((npad + 2 * h->halo) * sizeof(float));
  const size_t head_h = head + 2 * (vech - vec) + (ir ? 3 * (vecfh - vecf) : 0);
  cudaError_t e = cudaMalloc(&h->mem, head_h + vbytes + cbytes + tbytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(sparse)");
  char* p = static_cast<char*>(h->mem);
  auto take = [&p](size_t bytes) {
    char* at = p;
    p += bytes;
    return at;
  };
  h->soff = reinterpret_cast<int64_t*>(take(align_up((nslices + 1) * sizeof(int64_t))));
  h->c = reinterpret_cast<double*>(take(vec));
  h->xa = reinterpret_cast<double*>(take(vech)) + h->halo;
  h->xb = reinterpret_cast<double*>(take(vech)) + h->halo;
  h->xout = reinterpret_cast<double*>(take(vec));
  h->part = reinterpret_cast<double*>(take(align_up(2 * kMaxGrid * sizeof(double))));
  h->ctl = reinterpret_cast<Ctl*>(take(align_up(sizeof(Ctl))));
  unsigned long long* bmax = reinterpret_cast<unsigned long long*>(take(align_up(sizeof(unsigned long long))));
  if (keep_d) h->d = reinterpret_cast<double*>(take(vec));
  if (ir) {
    h->rf = reinterpret_cast<float*>(take(vecfh)) + h->halo;
    h->da = reinterpret_cast<float*>(take(vecfh)) + h->halo;
    h->db = reinterpret_cast<float*>(take(vecfh)) + h->halo;
  }
  h->sval = reinterpret_cast<double*>(take(vbytes));
  if (dia)
    h->doff = reinterpret_cast<int32_t*>(take(cbytes));
  else
    h->scol = reinterpret_cast<int32_t*>(take(cbytes));
  if (ir) h->tlo = take(tbytes);
  jacobi_csr* raw = h.get();
  auto fail = [&](cudaError_t err, const char* what) {
    cudaFree(raw->mem);
    raw->mem = nullptr;
    return cuda_fail(err, what);
  };
#define CSR_CK(call)                                 \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return fail(e_, #call);   \
  } while (0)
  CSR_CK(cudaMemsetAsync(h->mem, 0, head_h, s));
  CSR_CK(cudaMemcpyAsync(h->soff, hoff.data(), (nslices + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CSR_CK(cudaMemcpyAsync(h->c, d->B, n * sizeof(double), cudaMemcpyDefault, s));
  if (dia) {
    CSR_CK(cudaMemcpyAsync(h->doff, offs.data(), offs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CSR_CK(cudaMemsetAsync(h->sval, 0, vbytes, s));
    CSR_CK(launch_csr_dia_fill(n, rp, ci, va, dd, h->doff, h->ndiag, h->sval, h->c, bmax, s));
  } else {
    CSR_CK(launch_csr_fill(n, rp, ci, va, dd, h->soff, h->sval, h->scol, h->c, bmax, s));
  }
  if (keep_d) CSR_CK(cudaMemcpyAsync(h->d, dd, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (ir) {
    CSR_CK(launch_csr_narrow(d->precision == JACOBI_BF16_IR ? CsrInner::BF16 : CsrInner::F32, h->sval, stored, h->tlo,
                             s));
  }
  unsigned long long hb = 0;
  CSR_CK(cudaMemcpyAsync(&hb, bmax, sizeof(hb), cudaMemcpyDeviceToHost, s));
  CSR_CK(cudaStreamSynchronize(s));
  std::memcpy(&h->bnorm, &hb, sizeof(double));
#undef CSR_CK
  const int cap = ir ? csr_ir_max_grid(d->precision == JACOBI_BF16_IR ? CsrInner::BF16 : CsrInner::F32)
                     : csr_max_grid();
  if (cap <= 0) return fail(cudaGetLastError(), "occupancy query");
  const int64_t want = (nslices + csr_warps_per_cta() - 1) / csr_warps_per_cta();
  h->grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(cap, want)));
  *out = h.release();
  return JACOBI_OK;
}

}  // namespace

extern "C" {

void jacobi_desc_init(jacobi_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->nrhs = 1;
  d->precision = JACOBI_FP64;
  d->norm = JACOBI_NORM_INF;
}

int jacobi_workspace_size(const jacobi_desc* d, size_t* bytes) {
  if (!d || !bytes || d->n < 1 || d->nrhs < 1) return JACOBI_ERR_INVALID_ARG;
  const Layout L = make_layout(d->n, d->precision, !can_borrow(d), (d->flags & JACOBI_FLAG_SYMMETRIC) != 0);
  *bytes = d->nrhs > 1 ? mrhs_layout(L.total, d->n, L.ld, d->nrhs, (d->flags & JACOBI_FLAG_TC_RESIDUAL) != 0).total
                        : L.total;
  return JACOBI_OK;
}

int jacobi_setup_ex(const jacobi_desc* d, jacobi_handle** out) {
  if (!out) return JACOBI_ERR_INVALID_ARG;
  *out = nullptr;
  int st = validate_desc(d);
  if (st != JACOBI_OK) return st;
  const bool copy_A = !can_borrow(d);
  jacobi_handle* h = nullptr;
  st = make_handle(d, copy_A, &h);
  if (st != JACOBI_OK) return st;
  st = prepare(h, d->A, d->lda, d->B, copy_A);
  if (st == JACOBI_OK && h->nrhs > 1) st = mrhs_prepare(h, d->B, d->ldb);
  if (st != JACOBI_OK) {
    jacobi_destroy(h);
    return st;
  }
  *out = h;
  return JACOBI_OK;
}

int jacobi_setup(const double* A, const double* B, int64_t n, jacobi_handle** out) {
  if (!out) return JACOBI_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A || !B || n < 1) return JACOBI_ERR_INVALID_ARG;
  jacobi_desc d;
  jacobi_desc_init(&d);
  d.n = n;
  d.A = A;
  d.lda = n;
  d.B = B;
  d.ldb = n;
  d.flags = JACOBI_FLAG_COPY_A;
  jacobi_handle* h = nullptr;
  int st = make_handle(&d, true, &h);
  if (st != JACOBI_OK) return st;
  // host -> device: A straight into its padded place in the workspace, B into b
  double* A64 = h->at<double>(h->L.A64);
  double* b = h->at<double>(h->L.b);
  cudaError_t e = cudaMemcpy2DAsync(A64, h->L.ld * sizeof(double), A, n * sizeof(double), n * sizeof(double), n,
                                    cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b, B, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) {
    jacobi_destroy(h);
    return cuda_fail(e, "host-to-device copy of A, B");
  }
  st = prepare(h, A64, h->L.ld, b, true);
  if (st != JACOBI_OK) {
    jacobi_destroy(h);
    return st;
  }
  *out = h;
  return JACOBI_OK;
}

int jacobi_solve_async(jacobi_handle* h, const double* X0, int64_t max_iter, double tol, double* X_out,
                       jacobi_stats* stats_dev) {
  if (!h || !X_out || max_iter < 1 || !(tol > 0.0) || !std::isfinite(tol)) return JACOBI_ERR_INVALID_ARG;
  if (h->nrhs > 1) return JACOBI_ERR_UNSUPPORTED;  // many right-hand sides: jacobi_solve_ex
  if (h->symmetric) return sym_solve(h, X0, max_iter, tol, X_out, stats_dev);  // host-driven: returns when done
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  CK(cudaMemsetAsync(h->at<char>(h->L.ctl), 0, sizeof(Ctl), s));
  if (X0) {
    CK(cudaMemcpyAsync(h->at<double>(h->L.xa), X0, n * sizeof(double), cudaMemcpyDefault, s));
    if (h->split_residual)
      CK(launch_split_x(h->at<double>(h->L.xa), n, h->at<unsigned long long>(h->L.cmax), h->at<float2>(h->L.xsa), s));
  } else {
    CK(cudaMemsetAsync(h->at<char>(h->L.xa), 0, n * sizeof(double), s));
  }
  SolveParams p{};
  p.n = n;
  p.A = h->A64;
  p.lda = h->lda64;
  p.Nlow = h->precision != JACOBI_FP64 ? h->at<void>(h->L.Nlow) : nullptr;
  p.ldn = h->L.ld;
  p.Nlow_w = h->precision != JACOBI_FP64 ? h->at<void>(h->L.Nlow) : nullptr;
  p.nready = h->fuse_narrow ? h->at<int>(h->L.nready) : nullptr;
  p.rowfac_w = h->at<float>(h->L.rowfac);
  p.b = h->at<double>(h->L.b);
  p.d = h->at<double>(h->L.d);
  p.rinv = h->at<double>(h->L.rinv);
  p.rowfac = h->at<float>(h->L.rowfac);
  p.bnorm = h->at<double>(h->L.bnorm);
  p.xa = h->at<double>(h->L.xa);
  p.xb = h->at<double>(h->L.xb);
  p.xsa = h->split_residual ? h->at<float2>(h->L.xsa) : nullptr;
  p.xsb = h->split_residual ? h->at<float2>(h->L.xsb) : nullptr;
  p.c1 = h->at<float>(h->L.c1);
  p.da = h->at<float>(h->L.da);
  p.db = h->at<float>(h->L.db);
  p.part = h->at<double>(h->L.part);
  p.ctl = h->at<Ctl>(h->L.ctl);
  p.x_out = X_out;
  p.stats_out = stats_dev;
  p.max_iter = max_iter;
  p.tol = tol;
  p.norm = h->norm;
  p.x0_zero = X0 ? 0 : 1;
  p.max_outer = h->max_outer;
  p.max_inner = h->max_inner;
  p.inner_rtol = h->inner_rtol;
  p.rexp = h->split_residual ? h->at<int>(h->L.rexp) : nullptr;
  p.cmax = h->at<unsigned long long>(h->L.cmax);
  p.wait_ns = h->wait_ns;
  p.test_drop_copy = h->test_drop_copy;
  cudaError_t e;
  if (h->method == JACOBI_METHOD_SOR) {
    CK(cudaMemsetAsync(h->at<char>(h->L.gsflags), 0, kMaxGrid * sizeof(int), s));
    CK(cudaMemsetAsync(h->at<char>(h->L.gsmbox), 0xFF, 2 * static_cast<size_t>(n) * sizeof(double), s));
    GsParams g{};
    g.n = n;
    g.A = h->A64;
    g.lda = h->lda64;
    g.b = p.b;
    g.d = p.d;
    g.rinv = p.rinv;
    g.xa = p.xa;
    g.xb = p.xb;
    g.flags = h->at<int>(h->L.gsflags);
    g.mbox = h->at<unsigned long long>(h->L.gsmbox);
    g.part = p.part;
    g.ctl = p.ctl;
    g.x_out = X_out;
    g.stats_out = stats_dev;
    g.max_iter = max_iter;
    g.tol = tol;
    g.norm = h->norm;
    g.omega = h->omega;
    g.cmax = h->at<unsigned long long>(h->L.cmax);
    g.rexp = h->at<int>(h->L.rexp);
    g.test_skip_publish = h->test_skip_arrival;
    g.wait_ns = h->wait_ns;
    e = launch_gs_solve(g, h->grid, s);
  } else {
    e = h->precision == JACOBI_FP64 ? launch_fp64_solve(p, h->grid, s)
                                    : launch_ir_solve(narrow_kind(h->precision), p, h->grid, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch");
  return JACOBI_OK;
}

int jacobi_last_stats(jacobi_handle* h, jacobi_stats* stats) {
  if (!h || !stats) return JACOBI_ERR_INVALID_ARG;
  Ctl* ctl = h->at<Ctl>(h->L.ctl);
  CK(cudaMemcpyAsync(stats, &ctl->result, sizeof(jacobi_stats), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return JACOBI_OK;
}

int jacobi_solve_ex(jacobi_handle* h, const double* X0, int64_t max_iter, double tol, double* X_out,
                    jacobi_stats* stats) {
  if (h && h->nrhs > 1) {
    if (!X_out || max_iter < 1 || !(tol > 0.0) || !std::isfinite(tol)) return JACOBI_ERR_INVALID_ARG;
    return mrhs_solve(h, X0, max_iter, tol, X_out, stats);
  }
  int st = jacobi_solve_async(h, X0, max_iter, tol, X_out, nullptr);
  if (st != JACOBI_OK) return st;
  jacobi_stats local;
  st = jacobi_last_stats(h, &local);
  if (st != JACOBI_OK) return st;
  if (stats) *stats = local;
  return local.status;
}

int jacobi_solve(jacobi_handle* h, const double* X0, int64_t max_iter, double tol, double* X_out,
                 int64_t* iters_out, double* final_delta_out) {
  if (!h || !X_out) return JACOBI_ERR_INVALID_ARG;
  if (h->nrhs > 1) return JACOBI_ERR_UNSUPPORTED;
  double* xout = h->at<double>(h->L.xout);
  int st = jacobi_solve_async(h, X0, max_iter, tol, xout, nullptr);
  if (st != JACOBI_OK) return st;
  jacobi_stats local;
  Ctl* ctl = h->at<Ctl>(h->L.ctl);
  CK(cudaMemcpyAsync(&local, &ctl->result, sizeof(local), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(X_out, xout, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (iters_out) *iters_out = local.sweeps;
  if (final_delta_out) *final_delta_out = local.final_delta;
  return local.status;
}

int jacobi_column_stats(jacobi_handle* h, int64_t* iters, double* value) {
  if (!h || h->nrhs < 2) return JACOBI_ERR_INVALID_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  const size_t r = static_cast<size_t>(h->nrhs);
  for (size_t c = 0; c < r; ++c) {
    if (iters) iters[c] = c < h->col_iters.size() ? h->col_iters[c] : 0;
    if (value) value[c] = c < h->col_value.size() ? h->col_value[c] : std::nan("");
  }
  return JACOBI_OK;
}

int jacobi_residual(jacobi_handle* h, const double* X, double* rel_out) {
  if (!h || !X || !rel_out) return JACOBI_ERR_INVALID_ARG;
  unsigned long long* bits = h->at<unsigned long long>(h->L.keys) + 1;
  CK(cudaMemsetAsync(bits, 0, sizeof(unsigned long long), h->stream));
  CK(launch_residual(h->A64, h->lda64, h->n, h->at<double>(h->L.b), X, bits, h->stream));
  unsigned long long host[1];
  double bn = 0.0;
  CK(cudaMemcpyAsync(host, bits, sizeof(host), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&bn, h->at<double>(h->L.bnorm), sizeof(bn), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  double rmax;
  std::memcpy(&rmax, host, sizeof(rmax));
  *rel_out = rmax / bn;
  return JACOBI_OK;
}

int jacobi_get_narrow(jacobi_handle* h, void* dst_host, int64_t ld_dst, float* scale_host) {
  if (!h || !dst_host || ld_dst < h->n || h->precision == JACOBI_FP64) return JACOBI_ERR_INVALID_ARG;
  if (h->symmetric) return JACOBI_ERR_UNSUPPORTED;  // packed upper tiles, not a row-major copy
  const size_t es = narrow_size(h->precision);
  if (h->fuse_narrow) {  // not written yet if no solve has run an inner sweep: write it now
    int ready = 0;
    CK(cudaMemcpyAsync(&ready, h->at<int>(h->L.nready), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (!ready) CK(write_narrow(h));
  }
  CK(cudaMemcpy2DAsync(dst_host, ld_dst * es, h->at<char>(h->L.Nlow), h->L.ld * es, h->n * es, h->n,
                       cudaMemcpyDeviceToHost, h->stream));
  if (scale_host) {
    if (h->precision == JACOBI_FP8_IR) {
      CK(cudaMemcpyAsync(scale_host, h->at<float>(h->L.scale), h->n * sizeof(float), cudaMemcpyDeviceToHost,
                         h->stream));
    } else {
      for (int64_t i = 0; i < h->n; ++i) scale_host[i] = 1.0f;
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  return JACOBI_OK;
}

int jacobi_last_trace(jacobi_handle* h, int64_t* t_end_ns, int32_t* kinds, int32_t cap, int32_t* count) {
  if (!h || !count || cap < 0 || (cap > 0 && (!t_end_ns || !kinds))) return JACOBI_ERR_INVALID_ARG;
  if (h->nrhs > 1 || h->symmetric) {  // host-driven path: CUDA-event timeline
    const int32_t m = static_cast<int32_t>(h->htrace_kind.size());
    *count = m;
    for (int32_t i = 0; i < m && i < cap; ++i) {
      t_end_ns[i] = h->htrace_end[static_cast<size_t>(i)];
      kinds[i] = h->htrace_kind[static_cast<size_t>(i)];
    }
    return JACOBI_OK;
  }
  Ctl* ctl = h->at<Ctl>(h->L.ctl);
  Ctl* host = static_cast<Ctl*>(std::malloc(sizeof(Ctl)));
  if (!host) return JACOBI_ERR_OUT_OF_MEMORY;
  cudaError_t e = cudaMemcpyAsync(host, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    std::free(host);
    return cuda_fail(e, "trace read");
  }
  *count = host->nphase;
  const int m = host->nphase < cap ? host->nphase : cap;
  for (int i = 0; i < m; ++i) {
    t_end_ns[i] = static_cast<int64_t>(host->t_end[i] - host->t_start);
    kinds[i] = host->kind[i];
  }
  std::free(host);
  return JACOBI_OK;
}

void jacobi_destroy(jacobi_handle* h) {
  if (!h) return;
  if (h->own_ws && h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
  }
  delete h;
}

const char* jacobi_status_string(int status) {
  switch (status) {
    case JACOBI_OK: return "converged";
    case JACOBI_NOT_CONVERGED: return "iteration limit reached without convergence";
    case JACOBI_ERR_INVALID_ARG: return "invalid argument";
    case JACOBI_ERR_ZERO_DIAGONAL: return "zero diagonal entry (a_ii == 0)";
    case JACOBI_ERR_NONFINITE: return "non-finite value (diagonal or iterate)";
    case JACOBI_ERR_OUT_OF_MEMORY: return "out of device memory or workspace too small";
    case JACOBI_ERR_CUDA: return "CUDA runtime error";
    case JACOBI_ERR_TIMEOUT: return "device-side wait timed out";
    case JACOBI_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

const char* jacobi_last_cuda_error(void) { return g_cuda_err; }


int jacobi_csr_setup(const jacobi_csr_desc* d, jacobi_csr** out) { return csr_setup(d, out); }

int jacobi_csr_solve_async(jacobi_csr* h, const double* X0, int64_t max_iter, double tol, double* X_out) {
  if (!h || !X_out || max_iter < 1 || !(tol > 0.0) || !std::isfinite(tol)) return JACOBI_ERR_INVALID_ARG;
  cudaStream_t s = h->stream;
  CK(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), s));
  if (X0)
    CK(cudaMemcpyAsync(h->xa, X0, h->n * sizeof(double), cudaMemcpyDefault, s));
  else
    CK(cudaMemsetAsync(h->xa, 0, h->n * sizeof(double), s));
  CsrParams p{};
  p.n = h->n;
  p.nslices = h->nslices;
  p.soff = h->soff;
  p.sval = h->sval;
  p.scol = h->scol;
  p.c = h->c;
  p.xa = h->xa;
  p.xb = h->xb;
  p.part = h->part;
  p.ctl = h->ctl;
  p.x_out = is_device_memory(X_out) ? X_out : h->xout;
  p.stats_out = nullptr;
  p.max_iter = max_iter;
  p.tol = tol;
  p.norm = h->norm;
  p.d = h->d;
  p.bnorm = h->bnorm;
  p.test_skip_arrival = h->test_skip_arrival;
  p.wait_ns = h->wait_ns;
  p.doff = h->doff;
  p.ndiag = h->ndiag;
  cudaError_t e;
  if (h->precision == JACOBI_FP64) {
    e = launch_csr_solve(p, h->grid, s);
  } else {
    CsrIrParams q{};
    q.base = p;
    q.tlo = h->tlo;
    q.rf = h->rf;
    q.da = h->da;
    q.db = h->db;
    q.inner_rtol = h->inner_rtol;
    q.max_inner = h->max_inner;
    q.max_outer = h->max_outer;
    e = launch_csr_ir_solve(h->precision == JACOBI_BF16_IR ? CsrInner::BF16 : CsrInner::F32, q, h->grid, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch (sparse)");
  if (p.x_out != X_out) CK(cudaMemcpyAsync(X_out, h->xout, h->n * sizeof(double), cudaMemcpyDefault, s));
  return JACOBI_OK;
}

int jacobi_csr_last_stats(jacobi_csr* h, jacobi_stats* stats) {
  if (!h || !stats) return JACOBI_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(stats, &h->ctl->result, sizeof(jacobi_stats), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return JACOBI_OK;
}

int jacobi_csr_solve(jacobi_csr* h, const double* X0, int64_t max_iter, double tol, double* X_out,
                     jacobi_stats* stats) {
  int st = jacobi_csr_solve_async(h, X0, max_iter, tol, X_out);
  if (st != JACOBI_OK) return st;
  jacobi_stats local;
  st = jacobi_csr_last_stats(h, &local);
  if (st != JACOBI_OK) return st;
  if (stats) *stats = local;
  return local.status;
}

int jacobi_csr_info(jacobi_csr* h, int64_t* stored_slots, int64_t* slices, int32_t* grid) {
  if (!h) return JACOBI_ERR_INVALID_ARG;
  if (stored_slots) *stored_slots = h->stored;
  if (slices) *slices = h->nslices;
  if (grid) *grid = h->grid;
  return JACOBI_OK;
}

int jacobi_csr_format(jacobi_csr* h, int32_t* format, int32_t* ndiag) {
  if (!h) return JACOBI_ERR_INVALID_ARG;
  if (format) *format = h->ndiag > 0 ? JACOBI_CSR_DIA : JACOBI_CSR_ELL;
  if (ndiag) *ndiag = h->ndiag;
  return JACOBI_OK;
}

int jacobi_csr_last_trace(jacobi_csr* h, int64_t* t_end_ns, int32_t* kinds, int32_t cap, int32_t* count) {
  if (!h || !count || cap < 0 || (cap > 0 && (!t_end_ns || !kinds))) return JACOBI_ERR_INVALID_ARG;
  Ctl* host = static_cast<Ctl*>(std::malloc(sizeof(Ctl)));
  if (!host) return JACOBI_ERR_OUT_OF_MEMORY;
  cudaError_t e = cudaMemcpyAsync(host, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    std::free(host);
    return cuda_fail(e, "trace read");
  }
  *count = host->nphase;
  const int m = host->nphase < cap ? host->nphase : cap;
  for (int i = 0; i < m; ++i) {
    t_end_ns[i] = static_cast<int64_t>(host->t_end[i] - host->t_start);
    kinds[i] = host->kind[i];
  }
  std::free(host);
  return JACOBI_OK;
}

void jacobi_csr_destroy(jacobi_csr* h) {
  if (!h) return;
  if (h->mem) cudaFree(h->mem);
  delete h;
}

}  // extern "C"
