"""GB300-native MC-PDIPM hot path (Yamashita & Nakata, matrix-completion primal-dual
interior-point method): libmcsdp (CUDA, sm_103a) behind a C ABI, with a thin Python binding.

    from paper_1310_6919_gb300 import Problem
"""
from .binding import (Problem, MCSDPError, build_library, solve_batch, gemm_tc, tune,
                      tune_cache_clear)

__all__ = ["Problem", "MCSDPError", "build_library", "solve_batch", "gemm_tc", "tune",
           "tune_cache_clear"]
