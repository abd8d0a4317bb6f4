"""GB300 inverse ray-shooting for microlensing magnification maps
(arXiv:2204.10871).

The compute path is the CUDA library built from csrc/ (see build.py); this
package holds its ctypes binding (irs.py, same names as the C ABI in
include/irs.h) and a seeded synthetic lens generator (lensgen.py).  Importing
the package does not load the library; the first call does, and fails loudly
if it has not been built.
"""
from .irs import (IRS_BRUTE, IRS_INTERP, IRS_MLP, IRS_PLANE_CIRCLE, IRS_PLANE_RECT, IrsError,
                  IrsMlpReport, IrsParams, IrsPlanInfo, IrsTimings, IrsTuneResult, Plan, irs_autotune,
                  irs_magnify, irs_mlp_forward, irs_mlp_grad, irs_mlp_params, irs_mlp_train, irs_make_map,
                  irs_make_map_brute_noalloc, irs_make_map_rows, irs_make_maps_batched, irs_plan, irs_plan_destroy,
                  irs_plan_info_get, irs_plan_set_timing, irs_plan_sync, irs_plan_timings,
                  irs_shoot_rays, irs_status_str, make_params)

__all__ = ["IRS_BRUTE", "IRS_INTERP", "IRS_MLP", "IRS_PLANE_CIRCLE", "IRS_PLANE_RECT", "IrsError",
           "IrsMlpReport", "IrsParams", "IrsPlanInfo", "IrsTimings", "IrsTuneResult", "Plan",
           "irs_autotune", "irs_magnify", "irs_mlp_forward", "irs_mlp_grad", "irs_mlp_params",
           "irs_mlp_train", "irs_make_map",
           "irs_make_map_brute_noalloc", "irs_make_map_rows", "irs_make_maps_batched", "irs_plan", "irs_plan_destroy",
           "irs_plan_info_get", "irs_plan_set_timing", "irs_plan_sync", "irs_plan_timings",
           "irs_shoot_rays", "irs_status_str", "make_params"]
