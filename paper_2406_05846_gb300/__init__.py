"""GB300-native STROM: sparse moment relaxation + batched sGS-ADMM on sm_103a.

The compute path is libstrom.so (C ABI in include/strom.h): a host C++
relaxation builder and hand-written CUDA kernels. This package is the thin
Python binding; it has no CPU fallback.
"""
from ._native import (STROM_ERR_CUDA, STROM_ERR_INVALID, STROM_ERR_NOT_PD, STROM_ERR_NUMERICAL, STROM_ERR_OOM,
                      STROM_ERR_TIMEOUT, STROM_FACTOR_AUTO, STROM_FACTOR_DENSE, STROM_FACTOR_SPARSE, STROM_MAXITER,
                      STROM_OK, STROM_PREC_FP32, STROM_PREC_FP64, STROM_PREC_MIXED, StromError, lib)
from .api import (Batch, Certificate, Problem, PsdPlan, Result, Sdp, Server, Solver, WarmStore, certify_host,
                  default_options,
                  kernel_psd_project, kernel_spmv_csr, launch_count, moment_rank_test, transfer_bytes, warm_select)

__all__ = ["lib", "Batch", "Server", "Problem", "Sdp", "Solver", "PsdPlan", "Result", "Certificate", "default_options",
           "kernel_psd_project", "kernel_spmv_csr", "certify_host", "launch_count", "WarmStore", "warm_select", "moment_rank_test", "transfer_bytes", "STROM_OK", "STROM_MAXITER", "STROM_PREC_FP64", "STROM_PREC_FP32",
           "STROM_PREC_MIXED", "STROM_FACTOR_AUTO", "STROM_FACTOR_DENSE", "STROM_FACTOR_SPARSE",
           "STROM_ERR_INVALID", "STROM_ERR_OOM", "STROM_ERR_NOT_PD", "STROM_ERR_NUMERICAL", "STROM_ERR_TIMEOUT",
           "STROM_ERR_CUDA", "StromError"]
