"""ctypes loader of libsie.so (the C ABI declared in include/sie.h).

The library is built in-tree by paper_2210_04891_gb300.build (or
__graft_entry__.build()).  There is no fallback: if the library is missing or
fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsie.so")

SIE_OK = 0
ERRORS = {-1: "SIE_ERR_ARG", -2: "SIE_ERR_NONMANIFOLD", -3: "SIE_ERR_BAD_PORT", -4: "SIE_ERR_OOM",
          -5: "SIE_ERR_CUDA", -6: "SIE_ERR_NOT_CONVERGED", -7: "SIE_ERR_BREAKDOWN", -8: "SIE_ERR_TIMEOUT"}
SPACE_LOOP, SPACE_BRANCH = 0, 1
PREC_FP64, PREC_MIXED, PREC_DF = 0, 1, 2   # PREC_DF: double-float on the FP32 pipes (FP64-class)
REFINE_OFF, REFINE_FP64, REFINE_DF = 0, 1, 2   # sie_solve_opts.refine
KERNEL_STATIC, KERNEL_LOSSY = 0, 1
PC_AUTO, PC_BAND, PC_ND = 0, 1, 2

# every symbol include/sie.h declares
EXPORTS = ["sie_mesh_load", "sie_mesh_load_file", "sie_mesh_destroy", "loop_basis_build", "sie_loops_destroy", "sie_loops_export",
           "pfft_plan_create", "pfft_plan_destroy", "pfft_matvec", "pfft_precond_apply", "sie_solve",
           "pfft_plan_info", "pfft_plan_export", "pfft_convolve", "pfft_convolve_lossy", "pfft_convolve_noalloc", "pfft_profile_enable", "pfft_profile_read",
           "pfft_plan_launches", "pfft_plan_set_surface_model", "sie_postprocess", "sie_batch_create", "sie_batch_destroy",
           "sie_batch_matvec", "sie_batch_stats", "sie_batch_solve", "sie_batch_solve_graph", "pfft_precond_info",
           "pfft_precond_set_method", "pfft_precond_nd_info",
           "pfft_plan_set_kernel_tuning", "pfft_plan_get_kernel_tuning", "pfft_autotune_kernels", "pfft_autotune", "sie_mlp_create", "sie_mlp_destroy",
           "sie_mlp_param_count", "sie_mlp_get_params", "sie_mlp_set_params", "sie_mlp_forward", "sie_mlp_grad",
           "sie_mlp_train", "pfft_branch_features", "pfft_branch_probe_target", "pfft_plan_set_learned",
           "sie_selftest_bounded_wait", "sie_last_error"]
STAGES = ["loop_to_branch", "point_currents", "project", "fft_x_fwd", "fft_yz", "fft_x_inv", "interp",
          "near", "branch_to_loop", "precond_apply", "precond_factor", "arnoldi"]
(EXPORT_NEAR_PTR, EXPORT_NEAR_COL, EXPORT_LD, EXPORT_LDIRECT, EXPORT_HHAT, EXPORT_START, EXPORT_PROJ_PTR,
 EXPORT_PROJ_NODE, EXPORT_PROJ_W) = range(9)


class SiePort(ctypes.Structure):
    _fields_ = [("src", ctypes.POINTER(ctypes.c_int32)), ("n_src", ctypes.c_int32),
                ("sink", ctypes.POINTER(ctypes.c_int32)), ("n_sink", ctypes.c_int32)]


class SieLoopStats(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_branches", ctypes.c_int64), ("n_comp", ctypes.c_int64),
                ("n_loops", ctypes.c_int64), ("n_ports", ctypes.c_int64), ("tree_depth", ctypes.c_int64),
                ("nnz_A", ctypes.c_int64)]


class PfftParams(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32 * 3), ("order", ctypes.c_int32), ("near_factor", ctypes.c_double),
                ("near_min_diam", ctypes.c_double), ("n_touch", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("h0", ctypes.c_double)]


class KernelTuning(ctypes.Structure):
    _fields_ = [("near", ctypes.c_int32), ("far_slab", ctypes.c_int32), ("proj_slab", ctypes.c_int32),
                ("plane_gpc", ctypes.c_int32)]


class KernelTuneReport(ctypes.Structure):
    _fields_ = [("n_tried", ctypes.c_int32), ("best", ctypes.c_int32), ("cand", KernelTuning * 32),
                ("ms", ctypes.c_double * 32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("prec", ctypes.c_int32), ("refine", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations_max", ctypes.c_int32), ("iterations_sum", ctypes.c_int32),
                ("n_not_converged", ctypes.c_int32), ("residual_max", ctypes.c_double),
                ("seconds", ctypes.c_double), ("matvecs", ctypes.c_int64)]


class TuneReport(ctypes.Structure):
    _fields_ = [("n_tried", ctypes.c_int32), ("best", ctypes.c_int32), ("grid", (ctypes.c_int32 * 3) * 8),
                ("ms", ctypes.c_double * 8), ("err", ctypes.c_double * 8)]


class SieError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsie.so is not built ({LIB_PATH}); run paper_2210_04891_gb300.build.build() "
                          "or __graft_entry__.build() first")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    L.sie_mesh_load.argtypes = [P, I64, P, I64, P, P, I32, PP]
    L.sie_mesh_load_file.argtypes = [ctypes.c_char_p, PP]
    L.sie_mesh_destroy.argtypes = [P]
    L.loop_basis_build.argtypes = [P, ctypes.POINTER(SiePort), I32, PP, ctypes.POINTER(SieLoopStats)]
    L.sie_loops_destroy.argtypes = [P]
    L.sie_loops_export.argtypes = [P, P, P, P, P]
    L.pfft_plan_create.argtypes = [P, P, ctypes.POINTER(PfftParams), P, PP]
    L.pfft_plan_destroy.argtypes = [P]
    L.pfft_matvec.argtypes = [P, P, P, I32, P, I32, I32, P]
    L.pfft_precond_apply.argtypes = [P, P, P, I32, P, I32, P]
    L.sie_solve.argtypes = [P, P, I32, P, I32, ctypes.POINTER(SolveOpts), P, ctypes.POINTER(SolveStats)]
    L.pfft_plan_info.argtypes = [P, P, P, P, P, P, P, P]
    L.pfft_plan_export.argtypes = [P, I32, P, I64]
    L.pfft_convolve.argtypes = [P, P, I32, I32, P]
    L.pfft_convolve_noalloc.argtypes = [P, P, I32, I32, P]
    L.pfft_convolve_lossy.argtypes = [P, P, I32, ctypes.c_double, ctypes.c_double, I32, P]
    L.pfft_profile_enable.argtypes = [P, I32]
    L.pfft_profile_read.argtypes = [P, P, P]
    L.pfft_plan_set_surface_model.argtypes = [P, P, I32]
    L.sie_postprocess.argtypes = [P, P, I32, P, I32, P, P, P, P]
    L.sie_batch_create.argtypes = [P, I32, PP]
    L.pfft_precond_info.argtypes = [P, P, P, P]
    L.pfft_precond_set_method.argtypes = [P, I32]
    L.pfft_plan_set_kernel_tuning.argtypes = [P, P]
    L.pfft_plan_get_kernel_tuning.argtypes = [P, P]
    L.pfft_autotune_kernels.argtypes = [P, I32, D, P, P, P]
    L.pfft_precond_nd_info.argtypes = [P, P, P, P, P, P]
    L.sie_mlp_create.argtypes = [I32, ctypes.c_uint64, PP]
    L.sie_mlp_destroy.argtypes = [P]
    L.sie_mlp_param_count.argtypes = [P]
    L.sie_mlp_param_count.restype = I64
    L.sie_mlp_get_params.argtypes = [P, P, I64]
    L.sie_mlp_set_params.argtypes = [P, P, I64]
    L.sie_mlp_forward.argtypes = [P, P, I64, P, P]
    L.sie_mlp_grad.argtypes = [P, P, P, I64, P, P, P]
    L.sie_mlp_train.argtypes = [P, P, P, I64, I32, ctypes.c_float, P, P]
    L.pfft_branch_features.argtypes = [P, ctypes.c_double, P, P]
    L.pfft_branch_probe_target.argtypes = [P, P, I32, ctypes.c_double, P, P]
    L.pfft_plan_set_learned.argtypes = [P, P]
    L.sie_selftest_bounded_wait.argtypes = [P, ctypes.c_double, P]
    L.pfft_autotune.argtypes = [P, P, ctypes.POINTER(PfftParams), I32, ctypes.c_double, ctypes.c_double, P,
                                ctypes.POINTER(PfftParams), ctypes.POINTER(TuneReport)]
    L.sie_batch_destroy.argtypes = [P]
    L.sie_batch_matvec.argtypes = [P, P, P, P, P, I32, I32, I32, P]
    L.sie_batch_stats.argtypes = [P, P, P]
    L.sie_batch_solve.argtypes = [P, P, P, P, P, ctypes.POINTER(SolveOpts), P, P]
    L.sie_batch_solve_graph.argtypes = [P, P, P, P, P, ctypes.POINTER(SolveOpts), P, P]
    L.pfft_plan_launches.argtypes = [P]
    L.pfft_plan_launches.restype = I64
    L.sie_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def check(rc):
    if rc != SIE_OK:
        raise SieError(rc, lib().sie_last_error().decode())
    return rc
