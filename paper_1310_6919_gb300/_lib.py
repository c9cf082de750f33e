"""ctypes declarations of the C ABI in include/mcsdp.h (argument marshalling only)."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmcsdp.so")


class Problem_t(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("form", C.c_int32),
                ("c", C.POINTER(C.c_double)), ("nnz", C.c_int64),
                ("mat", C.POINTER(C.c_int32)), ("row", C.POINTER(C.c_int32)),
                ("col", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double))]


class Options_t(C.Structure):
    _fields_ = [("beta", C.c_double), ("gamma", C.c_double), ("gap_tol", C.c_double),
                ("feas_tol", C.c_double), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("timeout_cycles", C.c_int64), ("device", C.c_int32), ("verbose", C.c_int32),
                ("panel_max", C.c_int32), ("group_max", C.c_int32),
                ("panel_budget_mb", C.c_double), ("profile", C.c_int32), ("relax", C.c_int32),
                ("solve_warps", C.c_int32), ("mixed_gap", C.c_double), ("root_rows", C.c_int32),
                ("tensor_cores", C.c_int32), ("mixed_asm_gap", C.c_double), ("graph", C.c_int32),
                ("scm_blocks", C.c_int32)]


class Work_t(C.Structure):
    _fields_ = [("flops", C.c_double * 16), ("bytes", C.c_double * 16)]


class Stats_t(C.Structure):
    _fields_ = [("launches", C.c_int64), ("count", C.c_int64 * 16), ("ms", C.c_double * 16)]


KCLASS = ["ychol", "alg1", "scm_panel", "scm_tile", "scm_chol", "sce_backsolve", "pmatrix",
          "primal_step", "dual_step", "other", "pmatrix_side", "scm_panel_side", "scm_chol32",
          "root_gemm"]


class SymInfo_t(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("nsuper", C.c_int32),
                ("ngroup", C.c_int32), ("max_nrow", C.c_int32), ("max_ncol", C.c_int32),
                ("tree_height", C.c_int32), ("nnz_layout", C.c_int64),
                ("nnz_lower_E", C.c_int64), ("nslot", C.c_int64), ("table_bytes", C.c_int64),
                ("ncomp", C.c_int32), ("scm_blocks", C.c_int32)]


class Result_t(C.Structure):
    _fields_ = [("pobj", C.c_double), ("dobj", C.c_double), ("gap", C.c_double),
                ("pinf", C.c_double), ("dinf", C.c_double), ("mu", C.c_double),
                ("iters", C.c_int32), ("status", C.c_int32), ("seconds", C.c_double),
                ("t_scm", C.c_double), ("t_chol", C.c_double), ("t_pmat", C.c_double),
                ("t_other", C.c_double), ("precision", C.c_int32),
                ("promoted_iter", C.c_int32), ("refine_steps", C.c_int32),
                ("assembly_iter", C.c_int32)]


class TuneInfo_t(C.Structure):
    _fields_ = [("group_max", C.c_int32), ("panel_max", C.c_int32), ("cached", C.c_int32),
                ("ncand", C.c_int32), ("ms_per_iter", C.c_double * 8), ("key", C.c_int64 * 3)]


STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_NOT_PD", 3: "ERR_MAXITER", 4: "ERR_STALL",
          5: "ERR_NUMERIC", 6: "ERR_CUDA", 7: "ERR_OOM", 8: "ERR_TIMEOUT", 9: "ERR_STATE"}

EXPORTED = ["mcsdp_default_options", "mcsdp_create", "mcsdp_destroy", "mcsdp_last_error",
            "mcsdp_workspace_size", "mcsdp_set_workspace", "mcsdp_sym_info_get",
            "mcsdp_sym_export", "mcsdp_solve", "mcsdp_set_iterate", "mcsdp_get_iterate",
            "mcsdp_scm_assemble", "mcsdp_newton_step", "mcsdp_factors", "mcsdp_backward",
            "mcsdp_stats_get", "mcsdp_stats_reset", "mcsdp_work_model", "mcsdp_sce_solve_noalloc",
            "mcsdp_solve_batch", "mcsdp_pivot_reciprocal", "mcsdp_chol_task_order",
            "mcsdp_gemm_tc_work_size", "mcsdp_gemm_tc", "mcsdp_tune_workspace_size",
            "mcsdp_tune", "mcsdp_tune_cache_clear", "mcsdp_chol_block_task_order"]

_lib = None


def load():
    """Loads the in-tree libmcsdp.so; raises if it is missing (there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libmcsdp.so not built ({LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    P, V = C.c_void_p, C.c_void_p
    dp = C.POINTER(C.c_double)
    L.mcsdp_default_options.argtypes = [C.POINTER(Options_t)]
    L.mcsdp_default_options.restype = None
    L.mcsdp_create.argtypes = [C.POINTER(Problem_t), C.POINTER(Options_t), V, C.POINTER(P)]
    L.mcsdp_create.restype = C.c_int
    L.mcsdp_destroy.argtypes = [P]
    L.mcsdp_destroy.restype = None
    L.mcsdp_last_error.argtypes = [P]
    L.mcsdp_last_error.restype = C.c_char_p
    L.mcsdp_workspace_size.argtypes = [P, C.POINTER(C.c_size_t)]
    L.mcsdp_set_workspace.argtypes = [P, V, C.c_size_t]
    L.mcsdp_sym_info_get.argtypes = [P, C.POINTER(SymInfo_t)]
    L.mcsdp_sym_export.argtypes = [P, V, V, V, V, V, V]
    L.mcsdp_solve.argtypes = [P, C.POINTER(Result_t)]
    L.mcsdp_set_iterate.argtypes = [P, V, V]
    L.mcsdp_get_iterate.argtypes = [P, V, V, V]
    L.mcsdp_scm_assemble.argtypes = [P, V, V, V, C.c_int64, V, C.c_int32]
    L.mcsdp_newton_step.argtypes = [P, V, V, V, V, V, dp, dp, dp]
    L.mcsdp_factors.argtypes = [P, V, V, V, V]
    L.mcsdp_backward.argtypes = [P, V, V, V, V, V]
    L.mcsdp_stats_get.argtypes = [P, C.POINTER(Stats_t)]
    L.mcsdp_stats_reset.argtypes = [P]
    L.mcsdp_work_model.argtypes = [P, C.POINTER(Work_t)]
    L.mcsdp_sce_solve_noalloc.argtypes = [V, C.c_int64, V, V, C.c_int32, V]
    L.mcsdp_pivot_reciprocal.argtypes = [V, V, C.c_int64, V]
    L.mcsdp_chol_task_order.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_int64), V]
    L.mcsdp_chol_block_task_order.argtypes = [C.c_int32, V, C.POINTER(C.c_int64), V]
    L.mcsdp_solve_batch.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_int32,
                                    C.POINTER(Result_t)]
    L.mcsdp_gemm_tc_work_size.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]
    L.mcsdp_gemm_tc.argtypes = [C.c_int32, C.c_int32, C.c_int32, V, C.c_int64, V, C.c_int64, V,
                                C.c_int64, C.c_float, C.c_float, V, C.c_size_t, V]
    L.mcsdp_tune_workspace_size.argtypes = [C.POINTER(Problem_t), C.POINTER(Options_t),
                                            C.POINTER(C.c_size_t)]
    L.mcsdp_tune.argtypes = [C.POINTER(Problem_t), C.POINTER(Options_t), V, V, V, C.c_size_t,
                             C.c_int32, C.POINTER(TuneInfo_t)]
    L.mcsdp_tune_cache_clear.argtypes = []
    L.mcsdp_tune_cache_clear.restype = None
    for f in EXPORTED:
        if getattr(L, f).restype is C.c_int or f not in ("mcsdp_default_options", "mcsdp_destroy",
                                                           "mcsdp_last_error"):
            if f not in ("mcsdp_default_options", "mcsdp_destroy", "mcsdp_last_error",
                         "mcsdp_tune_cache_clear"):
                getattr(L, f).restype = C.c_int
    _lib = L
    return L
