"""GB300 engine for the Monte Carlo design objective of biomarker trials.

The compute path is libmcdesign (CUDA, sm_103a) behind the C ABI in
include/mcdesign.h; this package is its thin Python binding (ctypes) and the
build script.  Importing the package does not load the library; the first
call that needs it does, and raises when it is missing.
"""
from .binding import (MCD_ALL_BELOW, MCD_ANY_EXCEEDS, MCD_MAX_D, MCD_PLAN_AUTOTUNE, MCD_PLAN_FP64,
                      MCD_PLAN_GRAD, MCD_PLAN_GRAPH, Context, DeviceProblem, MCDError, Plan,
                      debug_normals, load, mc_design_eval, mc_design_eval_noalloc, mc_design_grad,
                      mc_fwer_calibrate, mc_smooth_argmax, mc_tps_argmax, mc_tps_fit, mc_tps_gcv, pipe_rates)

__all__ = ["Context", "DeviceProblem", "Plan", "MCDError", "load", "mc_design_eval", "mc_design_eval_noalloc",
           "mc_design_grad", "mc_fwer_calibrate", "mc_tps_fit", "mc_tps_argmax", "mc_tps_gcv",
           "mc_smooth_argmax", "debug_normals", "pipe_rates", "MCD_ANY_EXCEEDS", "MCD_ALL_BELOW", "MCD_MAX_D",
           "MCD_PLAN_GRAD", "MCD_PLAN_AUTOTUNE", "MCD_PLAN_GRAPH", "MCD_PLAN_FP64"]
