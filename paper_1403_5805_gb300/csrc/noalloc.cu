// jacobi_solve_fp64_noalloc: the FP64 solve without any device allocation.
//
// Some callers cannot allocate device memory while they run: a plugin inside a host application that
// owns the GPU's memory pool and forbids allocations outside it, or a latency-bound loop that cannot
// afford cudaMalloc's implicit synchronisation and its possible failure at run time.  This entry point
// serves them.  The caller passes A, B and X_out (its own device memory); every other buffer the
// persistent FP64 kernel needs (control block, iterate ping-pong, per-CTA partials, diagonal and its
// reciprocals) lives in one file-scope __device__ array of fixed size, so the call allocates nothing.
//
// The array exists once per device that loads this library and stays allocated until the process
// exits.  Every call shares it and it keeps the previous call's contents: whatever must start at zero
// (the control block, the diagonal-check key, ||B||) is cleared on the stream at the start of each call.
// Calls whose work overlaps on the GPU (different streams, or different host threads on one device)
// race on the array; serialise them.  The array's device address is looked up once per device and kept
// for the life of the process, so the call must not be used after cudaDeviceReset on that device (the
// reset unloads the module and the kept address goes stale).
#include <cmath>
#include <cstring>
#include <mutex>

#include "solver.cuh"

namespace jac {
namespace {

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Layout of the scratch array.
constexpr size_t kNaOffCtl = 0;
constexpr size_t kNaOffPart = align256(sizeof(Ctl));
constexpr size_t kNaOffKeys = kNaOffPart + align256(2 * kMaxGrid * sizeof(double));
constexpr size_t kNaOffBnorm = kNaOffKeys + 256;
constexpr size_t kNaOffD = kNaOffBnorm + 256;
constexpr size_t kNaVec = static_cast<size_t>(JACOBI_NOALLOC_MAX_N) * sizeof(double);
constexpr size_t kNaOffRinv = kNaOffD + kNaVec;
constexpr size_t kNaOffXa = kNaOffRinv + kNaVec;
constexpr size_t kNaOffXb = kNaOffXa + kNaVec;
constexpr size_t kNaBytes = kNaOffXb + kNaVec;

}  // namespace
}  // namespace jac

// The scratch of jacobi_solve_fp64_noalloc (about 1 MB).  In host code this name is only a host-side
// stand-in for the symbol: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[jac::kNaBytes];

namespace jac {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

bool device_memory(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace jac

using namespace jac;

extern "C" int jacobi_solve_fp64_noalloc(const double* A, int64_t lda, const double* B, int64_t n,
                                         const double* X0, int64_t max_iter, double tol, double* X_out,
                                         jacobi_stats* stats, void* stream) {
  if (!A || !B || !X_out || n < 1 || lda < n) return JACOBI_ERR_INVALID_ARG;
  if (n > JACOBI_NOALLOC_MAX_N) return JACOBI_ERR_INVALID_ARG;
  if (max_iter < 1 || !(tol > 0.0) || !std::isfinite(tol)) return JACOBI_ERR_INVALID_ARG;
  // rows are streamed in place by bulk copies: 16-byte aligned rows, and for odd n one padding element
  // per row is read (and ignored)
  if (reinterpret_cast<uintptr_t>(A) % 16 != 0 || lda % 2 != 0 || (n % 2 == 1 && lda == n))
    return JACOBI_ERR_INVALID_ARG;
  if (!device_memory(A) || !device_memory(B) || !device_memory(X_out) || (X0 && !device_memory(X0)))
    return JACOBI_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return JACOBI_ERR_CUDA;
  Ctl* ctl = reinterpret_cast<Ctl*>(base + kNaOffCtl);
  unsigned long long* key = reinterpret_cast<unsigned long long*>(base + kNaOffKeys);
  double* bnorm = reinterpret_cast<double*>(base + kNaOffBnorm);
  double* d = reinterpret_cast<double*>(base + kNaOffD);
  double* rinv = reinterpret_cast<double*>(base + kNaOffRinv);
  double* xa = reinterpret_cast<double*>(base + kNaOffXa);
  double* xb = reinterpret_cast<double*>(base + kNaOffXb);

#define NA_CK(call)                                      \
  do {                                                   \
    if ((call) != cudaSuccess) return JACOBI_ERR_CUDA;   \
  } while (0)
  // clear what must start at zero: the array keeps the previous call's contents
  NA_CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
  NA_CK(cudaMemsetAsync(key, 0xFF, sizeof(unsigned long long), s));
  NA_CK(cudaMemsetAsync(bnorm, 0, sizeof(double), s));
  NA_CK(launch_diag(A, lda, n, d, rinv, key, s));
  // b is read straight from the caller's B (the kernel only takes ||B|| when source == destination)
  NA_CK(launch_rhs(B, n, nullptr, const_cast<double*>(B), reinterpret_cast<unsigned long long*>(bnorm), nullptr, s));
  unsigned long long host_key = 0;
  NA_CK(cudaMemcpyAsync(&host_key, key, sizeof(host_key), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
  if (host_key != ~0ull) return (host_key & 0xFF) == 2 ? JACOBI_ERR_ZERO_DIAGONAL : JACOBI_ERR_NONFINITE;
  if (X0)
    NA_CK(cudaMemcpyAsync(xa, X0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else
    NA_CK(cudaMemsetAsync(xa, 0, n * sizeof(double), s));

  SolveParams p{};
  p.n = n;
  p.A = A;
  p.lda = lda;
  p.b = B;
  p.d = d;
  p.rinv = rinv;
  p.bnorm = bnorm;
  p.xa = xa;
  p.xb = xb;
  p.part = reinterpret_cast<double*>(base + kNaOffPart);
  p.ctl = ctl;
  p.x_out = X_out;
  p.stats_out = nullptr;
  p.max_iter = max_iter;
  p.tol = tol;
  p.norm = JACOBI_NORM_INF;
  p.x0_zero = X0 ? 0 : 1;
  p.wait_ns = 4000000000ull;
  int grid = max_coresident_grid(false, Narrow::F32);
  const int64_t want = (n + kRows - 1) / kRows;
  if (grid <= 0) return JACOBI_ERR_CUDA;
  if (want < grid) grid = static_cast<int>(want);
  if (grid > kMaxGrid) grid = kMaxGrid;
  NA_CK(launch_fp64_solve(p, grid, s));
  jacobi_stats local;
  NA_CK(cudaMemcpyAsync(&local, &ctl->result, sizeof(local), cudaMemcpyDeviceToHost, s));
  NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
  if (stats) *stats = local;
  return local.status;
}
