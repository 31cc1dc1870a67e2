"""GB300-native hybrid-dealiased FFT convolutions (Murasko & Bowman, arXiv 2303.17510).

The computation lives in libhd.so (hand-written CUDA for sm_103a behind the C
ABI of include/hd.h); this package is its thin Python binding.
"""
from ._binding import (DTYPE, KIND, MLP, MULT, PLAN_NO_WORK_BUFFER, SELECTOR_FEATURES, HdError, Plan, RaggedPlan, alu_peak, autotune, device_status,
                       dealias_bound, derive_params, enumerate_candidates, lib, make_desc, selector_choose,
                       selector_clear, selector_features, selector_install, status_string, tune_cache_clear,
                       tune_cache_get, tune_cache_put)

__all__ = ["DTYPE", "KIND", "MLP", "MULT", "PLAN_NO_WORK_BUFFER", "SELECTOR_FEATURES", "HdError", "Plan", "RaggedPlan", "alu_peak", "autotune", "dealias_bound", "derive_params", "device_status",
           "enumerate_candidates", "lib", "make_desc", "status_string", "tune_cache_clear", "tune_cache_get",
           "tune_cache_put", "selector_choose", "selector_clear", "selector_features", "selector_install"]
