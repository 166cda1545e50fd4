"""ctypes binding of libmf.so (argument marshalling only; all compute runs in the CUDA library)."""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmf.so")

MF_OK, MF_ERR_ARG, MF_ERR_CUDA, MF_ERR_OOM, MF_ERR_STATE, MF_ERR_NAN, MF_ERR_NOT_CONVERGED, \
    MF_ERR_BREAKDOWN, MF_ERR_ITER_LIMIT = range(9)
STATUS_NAMES = ["MF_OK", "MF_ERR_ARG", "MF_ERR_CUDA", "MF_ERR_OOM", "MF_ERR_STATE", "MF_ERR_NAN",
                "MF_ERR_NOT_CONVERGED", "MF_ERR_BREAKDOWN", "MF_ERR_ITER_LIMIT"]
MF_FP64, MF_FP32, MF_DF64 = 0, 1, 2
MF_PC_JACOBI, MF_PC_CHEBYSHEV, MF_PC_GMRES, MF_PC_MG = 0, 1, 2, 3
MF_SMOOTH_JACOBI, MF_SMOOTH_ASM = 0, 1

# every symbol include/mf.h declares
EXPORTS = ["mf_mesh_from_arrays", "mf_mesh_free", "mf_mesh_params_defaults", "mf_mesh_rotor_stator", "mf_mesh_sizes",
           "mf_mesh_read", "mf_mesh_interface", "mf_mortar_segments", "mf_mesh_coarsen_map", "mf_checkpoint_write", "mf_checkpoint_read", "mf_log_open", "mf_create", "mf_destroy", "mf_last_error", "mf_sizes",
           "mf_set_angle", "mf_node_coords", "mf_dirichlet", "mf_set_history", "mf_set_linearization",
           "mf_residual", "mf_apply_jacobian", "mf_diagonal", "mf_solver_defaults", "mf_solve_step",
           "mf_profile", "mf_profile_read", "mf_mg_attach", "mf_mg_prolongate", "mf_mg_restrict",
           "mf_mg_interpolate", "mf_solve_step_static", "mf_batch_create", "mf_batch_destroy",
           "mf_batch_apply_jacobian", "mf_batch_solve_step", "mf_batch_last_error", "mf_autotune", "mf_set_cells_per_block", "mf_kinetic_energy", "mf_energy", "mf_wall_loads", "mf_run_transient", "mf_fma_peak",
           "mf_mesh_slab", "mf_halo_pack", "mf_halo_add", "mf_mesh_from_arrays_ex",
           "mf_asm_setup", "mf_asm_apply", "mf_contract_probe", "mf_vec_dots", "mf_vec_maxpy", "mf_vec_axpby",
           "mf_vec_mul"]
PROF_KINDS = ["cell_jac_fp64", "cell_jac_fp32", "mortar_fp64", "mortar_fp32", "cell_residual",
              "cell_linearization", "dirichlet", "diagonal"]


class MfMeshParams(C.Structure):
    _fields_ = [("d", C.c_int), ("k", C.c_int), ("m", C.c_int), ("n_r", C.c_int), ("n_s", C.c_int),
                ("n_z", C.c_int), ("R", C.c_double), ("R_out", C.c_double), ("H", C.c_double), ("sq", C.c_double),
                ("phi0", C.c_double), ("blades", C.c_int), ("n_R_stator", C.c_int)]


class MfCheckpointInfo(C.Structure):
    _fields_ = [("bdf", C.c_int), ("step", C.c_int64), ("t", C.c_double), ("theta", C.c_double),
                ("dt", C.c_double), ("nu", C.c_double), ("omega", C.c_double)]


class MfOptions(C.Structure):
    _fields_ = [("penalty_F", C.c_double), ("reserved", C.c_int * 8)]


class MfSolverOpts(C.Structure):
    _fields_ = [("newton_rtol", C.c_double), ("newton_atol", C.c_double), ("max_newton", C.c_int),
                ("lin_rtol", C.c_double), ("restart", C.c_int), ("max_lin_iters", C.c_int),
                ("pc", C.c_int), ("pc_precision", C.c_int), ("cheb_degree", C.c_int),
                ("cheb_lo", C.c_double), ("theta", C.c_double), ("inner_iters", C.c_int),
                ("line_search", C.c_int), ("mg_smooth", C.c_int), ("mg_coarse_iters", C.c_int),
                ("deflate_pressure", C.c_int), ("use_graphs", C.c_int), ("outer_precision", C.c_int),
                ("batch_fallback", C.c_int), ("mg_smoother", C.c_int), ("step_rtol", C.c_double),
                ("smooth_cgs_passes", C.c_int)]


class MfSolveReport(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("lin_iters_total", C.c_int), ("lin_iters", C.c_int * 64),
                ("res_norm", C.c_double * 65), ("lambda_max", C.c_double), ("seconds", C.c_double),
                ("status", C.c_int), ("fallback_newton_iters", C.c_int),
                ("fallback_restarted", C.c_int)]


STEP_RECORD_FIELDS = ("kinetic_energy", "dissipation", "dissipation_sym", "torque_still", "torque_moving", "power",
                      "residual_reduction", "newton_iters")


class MfStepRecord(C.Structure):
    _fields_ = [(f, C.c_double) for f in STEP_RECORD_FIELDS]


class MfTuneResult(C.Structure):
    _fields_ = [("n_variants", C.c_int), ("cells_per_block", C.c_int * 3), ("ms", C.c_double * 3),
                ("chosen", C.c_int), ("from_cache", C.c_int)]


class MfProfile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 8), ("ms", C.c_double * 8)]


class MfSlabInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_cells", C.c_int64), ("layer_begin", C.c_int), ("layer_end", C.c_int),
                ("n_lo", C.c_int), ("n_hi", C.c_int)]


class MfError(RuntimeError):
    pass


_lib = None


def load():
    """Load libmf.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise MfError(f"{LIB_PATH} not built: run paper_2608_27423_b300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
    lib.mf_mesh_from_arrays.argtypes = [i32, i32, i64, vp, vp, vp, i64, vp, vp, dbl, i32, i32, dbl, dbl, vp, vp,
                                        C.POINTER(vp)]
    lib.mf_mesh_from_arrays_ex.argtypes = [i32, i32, i64, vp, vp, vp, i64, vp, vp, dbl, i32, i32, i32, dbl, dbl, vp,
                                           vp, C.POINTER(vp)]
    lib.mf_mesh_free.argtypes = [vp]
    lib.mf_mesh_free.restype = None
    lib.mf_mesh_params_defaults.argtypes = [C.POINTER(MfMeshParams)]
    lib.mf_mesh_params_defaults.restype = None
    lib.mf_mesh_rotor_stator.argtypes = [C.POINTER(MfMeshParams), C.POINTER(vp)]
    lib.mf_mesh_sizes.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), C.POINTER(i64), C.POINTER(i32),
                                  C.POINTER(i32)]
    lib.mf_mesh_read.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.mf_mesh_interface.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    lib.mf_mortar_segments.argtypes = [i32, i32, dbl, i32, vp, vp, vp, vp, C.POINTER(i32)]
    lib.mf_mesh_coarsen_map.argtypes = [C.POINTER(MfMeshParams), C.POINTER(MfMeshParams), vp, vp]
    lib.mf_log_open.argtypes = [C.c_char_p]
    lib.mf_checkpoint_write.argtypes = [C.c_char_p, vp, C.POINTER(MfCheckpointInfo), vp, vp]
    lib.mf_checkpoint_read.argtypes = [C.c_char_p, vp, C.POINTER(MfCheckpointInfo), vp, vp]
    lib.mf_create.argtypes = [vp, i32, dbl, dbl, dbl, i32, vp, C.POINTER(vp)]
    lib.mf_destroy.argtypes = [vp]
    lib.mf_last_error.argtypes = [vp]
    lib.mf_last_error.restype = C.c_char_p
    lib.mf_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    lib.mf_set_angle.argtypes = [vp, dbl, vp]
    lib.mf_node_coords.argtypes = [vp, vp, vp]
    lib.mf_dirichlet.argtypes = [vp, vp, vp]
    lib.mf_set_history.argtypes = [vp, vp, vp, vp]
    lib.mf_set_linearization.argtypes = [vp, vp, dbl, vp]
    lib.mf_residual.argtypes = [vp, vp, vp, vp]
    lib.mf_apply_jacobian.argtypes = [vp, vp, vp, i32, vp]
    lib.mf_diagonal.argtypes = [vp, vp, i32, vp]
    lib.mf_solver_defaults.argtypes = [C.POINTER(MfSolverOpts)]
    lib.mf_solver_defaults.restype = None
    lib.mf_solve_step.argtypes = [vp, vp, C.POINTER(MfSolverOpts), C.POINTER(MfSolveReport), vp]
    lib.mf_kinetic_energy.argtypes = [vp, vp, vp, vp]
    lib.mf_energy.argtypes = [vp, vp, vp, vp]
    lib.mf_wall_loads.argtypes = [vp, vp, vp, i32, vp, vp]
    lib.mf_run_transient.argtypes = [vp, vp, vp, i32, dbl, i32, i32, C.POINTER(MfSolverOpts), i32,
                                     C.POINTER(MfStepRecord), vp]
    lib.mf_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(vp)]
    lib.mf_batch_destroy.argtypes = [vp]
    lib.mf_batch_apply_jacobian.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), i32, vp]
    lib.mf_batch_solve_step.argtypes = [vp, C.POINTER(vp), C.POINTER(dbl), C.POINTER(MfSolverOpts), i32, i32, i32,
                                        C.POINTER(MfSolveReport), vp]
    lib.mf_autotune.argtypes = [vp, C.c_char_p, C.POINTER(MfTuneResult), vp]
    lib.mf_set_cells_per_block.argtypes = [vp, i32, i32]
    lib.mf_batch_last_error.argtypes = [vp]
    lib.mf_batch_last_error.restype = C.c_char_p
    lib.mf_solve_step_static.argtypes = [vp, vp, C.POINTER(MfSolverOpts), C.POINTER(MfSolveReport), vp]
    lib.mf_mg_attach.argtypes = [vp, vp, vp, vp]
    lib.mf_mg_prolongate.argtypes = [vp, vp, vp, vp]
    lib.mf_mg_restrict.argtypes = [vp, vp, vp, vp]
    lib.mf_mg_interpolate.argtypes = [vp, vp, vp, vp]
    lib.mf_profile.argtypes = [vp, i32]
    lib.mf_profile_read.argtypes = [vp, C.POINTER(MfProfile)]
    lib.mf_fma_peak.argtypes = [i32, C.POINTER(dbl), C.POINTER(dbl), vp]
    lib.mf_contract_probe.argtypes = [i32, i32, i32, vp, vp, vp, vp]
    lib.mf_vec_dots.argtypes = [i64, vp, i64, i32, vp, vp, vp, vp]
    lib.mf_vec_maxpy.argtypes = [i64, vp, i64, i32, vp, dbl, vp, vp]
    lib.mf_vec_axpby.argtypes = [i64, dbl, vp, dbl, vp, vp]
    lib.mf_vec_mul.argtypes = [i64, vp, vp, vp, vp]
    lib.mf_mesh_slab.argtypes = [vp, i32, i32, C.POINTER(vp), C.POINTER(MfSlabInfo), vp, vp, vp, vp, vp]
    lib.mf_halo_pack.argtypes = [vp, vp, i64, i32, vp, vp]
    lib.mf_asm_setup.argtypes = [vp, C.POINTER(i32), vp]
    lib.mf_asm_apply.argtypes = [vp, vp, vp, vp]
    lib.mf_halo_add.argtypes = [vp, vp, vp, i64, i32, vp, vp]
    for name in EXPORTS:
        f = getattr(lib, name)
        if name not in ("mf_mesh_free", "mf_last_error", "mf_batch_last_error", "mf_solver_defaults",
                        "mf_mesh_params_defaults"):
            f.restype = C.c_int
    _lib = lib
    return lib
