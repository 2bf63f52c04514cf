"""B300-native fixed-radius nearest-neighbour graph build (arXiv 2202.06929).

The CUDA kernels and the C ABI live in libfrnn.so (sources in csrc/, header in
include/frnn.h); this package is its Python binding plus the seeded input
generator used by the tests and the benchmark.
"""
from ._native import (ABI_FUNCTIONS, Csr, FrnnError, Plan, Server, plan_bytes, load, library_path, status_string,
                      version, FRNN_OK, FRNN_ERR_INVALID_ARG, FRNN_ERR_CUDA, FRNN_ERR_OOM,
                      FRNN_ERR_NONFINITE_INPUT, FRNN_ERR_TIMEOUT, FRNN_ERR_OVERFLOW,
                      FRNN_ERR_CAPACITY, FRNN_ERR_CHECK)

__all__ = ["ABI_FUNCTIONS", "Csr", "FrnnError", "Plan", "Server", "plan_bytes", "load", "library_path", "status_string",
           "version"]
