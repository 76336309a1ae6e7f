"""GB300-native (sm_103a) SiPO projection-LP solver.

The compute path is the CUDA library libsipo.so (C ABI in include/sipo.h);
this package only marshals arguments to it (`_abi`) and wraps the projector
pair as torch autograd functions (`autograd`).  `build()` compiles the
library in-tree.
"""
from ._abi import (SIPO_BF16, SIPO_CASE1, SIPO_CASE2, SIPO_F32, SIPO_F64, SIPO_GENERAL,
                   SIPO_ITER_LIMIT, SIPO_OPTIMAL, SIPO_PRIMAL_INFEASIBLE, Context, SipoError,
                   load, sipo_backproject, sipo_create, sipo_destroy, sipo_get_array,
                   sipo_kernel_launch_count, sipo_tile_count, sipo_profile, sipo_project, sipo_psf_apply,
                   sipo_psf_grad, sipo_set_psf_sigma, sipo_set_tolerances, sipo_get_trace, sipo_solve,
                   sipo_set_primal, sipo_set_primal_from, sipo_farkas_from, sipo_solve_probe, sipo_solve_race, sipo_solve_batched, sipo_warm_start,
                   sipo_create_bounded, sipo_response_map, sipo_response_metrics,
                   sipo_get_state, sipo_set_state)
from .build import build
from .two_stage import two_stage_solve
from .separation import case2_with_separation
from .response import (Richards, dose_to_response, response_case1, response_case2, response_general,
                       response_metrics, response_to_dose)

__all__ = [
    "build", "load", "Context", "SipoError", "sipo_create", "sipo_solve", "sipo_solve_batched",
    "sipo_warm_start", "sipo_set_primal", "sipo_set_primal_from", "sipo_farkas_from", "sipo_solve_probe", "sipo_solve_race", "sipo_get_state", "sipo_set_state", "two_stage_solve", "case2_with_separation",
    "sipo_create_bounded",
    "sipo_response_map", "sipo_response_metrics", "Richards", "response_to_dose", "dose_to_response",
    "response_case1", "response_case2", "response_general", "response_metrics",
    "sipo_project", "sipo_backproject", "sipo_psf_apply", "sipo_psf_grad", "sipo_set_psf_sigma",
    "sipo_get_array", "sipo_set_tolerances", "sipo_get_trace", "sipo_profile", "sipo_kernel_launch_count", "sipo_tile_count", "sipo_destroy",
    "SIPO_F32", "SIPO_F64", "SIPO_BF16", "SIPO_GENERAL", "SIPO_CASE1", "SIPO_CASE2",
    "SIPO_OPTIMAL", "SIPO_PRIMAL_INFEASIBLE", "SIPO_ITER_LIMIT",
]
