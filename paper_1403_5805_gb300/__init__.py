"""GB300-native Jacobi solver (dense, with a sparse CSR form) (Margaris, Souravlas & Roumeliotis, arXiv:1403.5805, Section 2).

The solver itself is the CUDA library ``_build/libjacobi.so`` (C ABI: ``include/jacobi.h``); this package
is its thin Python binding.  Build it with ``paper_1403_5805_gb300.build.build()``.
"""
from .binding import (BF16_IR, ERR_CUDA, ERR_INVALID_ARG, ERR_NONFINITE, ERR_OUT_OF_MEMORY, ERR_TIMEOUT,
                      ERR_UNSUPPORTED, ERR_ZERO_DIAGONAL, EXPORTS, FP8_IR, FP32_IR, FP64, LIB_PATH, NORM_2,
                      NORM_INF, NORM_RESID, NOT_CONVERGED, OK, DeviceSolver, HostSolver, JacobiDesc, JacobiError,
                      JacobiStats, load, BatchSolver, JacobiBatchDesc, MultiSolver, Server,
                      generate_request, CsrSolver, JacobiCsrDesc, batch_solve, measure_fma_rates)

__all__ = ["measure_fma_rates", "batch_solve", "CsrSolver", "JacobiCsrDesc", "Server", "generate_request", "MultiSolver", "BatchSolver", "JacobiBatchDesc", "DeviceSolver", "HostSolver", "JacobiDesc", "JacobiError", "JacobiStats", "load", "LIB_PATH", "EXPORTS",
           "OK", "NOT_CONVERGED", "ERR_INVALID_ARG", "ERR_ZERO_DIAGONAL", "ERR_NONFINITE", "ERR_OUT_OF_MEMORY",
           "ERR_CUDA", "ERR_TIMEOUT", "ERR_UNSUPPORTED", "FP64", "FP32_IR", "BF16_IR", "FP8_IR", "NORM_INF",
           "NORM_2", "NORM_RESID"]
