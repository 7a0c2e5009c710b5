"""GB300-native space-time least-squares solver for the Schroedinger equation.

A thin ctypes binding of the CUDA library `libstst.so` (C ABI declared in
include/stst.h). The functions keep the C names and only marshal arguments:
every numerical step runs in the library's CUDA kernels. PyTorch provides
device memory and streams. Importing works without a GPU; calling into the
library needs the built extension and raises if it is missing.
"""
from ._lib import (StstError, lib, library_path, stst_create, stst_create2, STST_FORM_LS, STST_FORM_UW,
                   stst_destroy, stst_strerror, stst_sizes, stst_quadrature_points, stst_assemble_1d,
                   stst_set_potential, stst_build_fd, stst_apply_sys, stst_apply_prec, stst_rhs,
                   stst_rhs_noalloc, stst_rhs_lift, stst_pcg_solve, stst_ir_solve, stst_profile, stst_profile_read,
                   stst_plan_info, stst_pcg_graph_info, stst_set_prec_operator, stst_batch_create, stst_batch_solve, stst_batch_destroy,
                   stst_set_autotune,
                   stst_set_time_solver, stst_set_fused_transforms, stst_fused_transforms_info, stst_fused_transforms_split,
                   stst_set_pencil, stst_pencil_info, stst_set_tensor_products, stst_tensor_products_info,
                   stst_set_geometry, stst_geometry_info, stst_set_fused_matvec, stst_persistent_solve,
                   stst_time_solver_info, stst_last_cuda_error, stst_tile_info, stst_ws_create,
                   stst_ws_destroy, stst_ws_num_params, stst_ws_get_params, stst_ws_set_params,
                   stst_ws_forward, stst_ws_set_output_scale, stst_ws_grad, stst_ws_train_step,
                   stst_pod_basis, stst_pod_project, stst_pod_expand, stst_pcg_solve_guarded, Problem,
                   stst_ws_whiten, stst_ws_target_scale, stst_ws_cascade,
                   STST_PREC_FP64, STST_PREC_FP32, STST_PREC_BF16, STST_OK, STST_NOT_CONVERGED, STST_BREAKDOWN,
                   STST_NOT_HPD, STST_TIMEOUT, STST_ERR_ARG, STST_ERR_HANDLE, STST_ERR_OOM, STST_ERR_CUDA,
                   STST_ERR_STATE)

__all__ = ["StstError", "lib", "library_path", "stst_create", "stst_create2", "STST_FORM_LS", "STST_FORM_UW",
           "stst_destroy", "stst_strerror", "stst_sizes", "stst_quadrature_points", "stst_assemble_1d",
           "stst_set_potential", "stst_build_fd", "stst_apply_sys", "stst_apply_prec", "stst_rhs",
           "stst_rhs_noalloc", "stst_rhs_lift", "stst_pcg_solve", "stst_ir_solve", "stst_profile", "stst_profile_read",
           "stst_plan_info", "stst_pcg_graph_info", "stst_set_prec_operator", "stst_batch_create", "stst_batch_solve", "stst_batch_destroy",
           "stst_set_autotune", "stst_set_time_solver", "stst_set_fused_transforms",
           "stst_fused_transforms_info", "stst_fused_transforms_split", "stst_set_pencil", "stst_pencil_info", "stst_set_tensor_products", "stst_set_geometry", "stst_set_fused_matvec",
           "stst_persistent_solve",
           "stst_geometry_info",
           "stst_tensor_products_info", "stst_time_solver_info", "stst_last_cuda_error", "stst_tile_info",
           "stst_ws_create", "stst_ws_destroy", "stst_ws_num_params", "stst_ws_get_params",
           "stst_ws_set_params", "stst_ws_forward", "stst_ws_set_output_scale", "stst_ws_grad",
           "stst_ws_train_step", "stst_pod_basis", "stst_pod_project", "stst_pod_expand",
           "stst_pcg_solve_guarded", "Problem", "stst_ws_whiten", "stst_ws_target_scale", "stst_ws_cascade", "STST_PREC_FP64", "STST_PREC_FP32", "STST_PREC_BF16", "STST_OK", "STST_NOT_CONVERGED", "STST_BREAKDOWN", "STST_NOT_HPD", "STST_TIMEOUT",
           "STST_ERR_ARG", "STST_ERR_HANDLE", "STST_ERR_OOM", "STST_ERR_CUDA", "STST_ERR_STATE"]
