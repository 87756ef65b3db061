// Symmetric A stored once for the narrow inner sweeps (sym.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "solver.cuh"

namespace jac {

constexpr int kSymTile = 128;  // rows and columns of a packed tile

// Tiles per side (ceil(n / 128)) and packed tiles on and above the diagonal (nt (nt + 1) / 2).
int64_t sym_tiles_per_side(int64_t n);
int64_t sym_tile_count(int64_t n);

// Packed upper tiles of A's off-diagonal part in the narrow type (FP32 or BF16; tile (I, J) at index
// I nt - I (I - 1) / 2 + (J - I), row-major 128 x 128), and rowfac_i = fl32(rinv_i).
cudaError_t launch_sym_pack(Narrow kind, const double* A, int64_t lda, int64_t n, const double* rinv, void* tiles,
                            float* rowfac, cudaStream_t s);
// One inner sweep: P (nt x nt x 128 floats) receives the tile partial sums, then dnew = c1 - rowfac * (P summed
// per row), xalt = xc + dnew, stats[0] = max |dnew - dcur| bits, stats[1] = max |dnew| bits (zeroed before).
cudaError_t launch_sym_sweep(Narrow kind, const void* tiles, int64_t n, const float* dcur, float* P, const float* c1,
                             const float* rowfac, float* dnew, const double* xc, double* xalt, unsigned long long* stats,
                             cudaStream_t s);
// FP64 residual of x (NULL: zero): c1 = d1 = fl32((b - A x) / a_ii), stats[0] = max |r| bits, stats[1] = max |c1|
// bits (zeroed before).
cudaError_t launch_sym_resid(int64_t n, const double* A, int64_t lda, const double* x, const double* b,
                             const double* rinv, float* c1, float* d1, unsigned long long* stats, cudaStream_t s);

}  // namespace jac
