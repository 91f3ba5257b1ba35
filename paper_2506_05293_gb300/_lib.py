"""ctypes declarations of the C ABI in include/lbm.h.

Loads ``libgb300lbm.so`` from this package directory.  There is no fallback:
if the library has not been built the import of the binding fails with an
error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_float, c_int, c_int32, c_int64,
                    c_size_t, c_uint8, c_uint64, c_void_p)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgb300lbm.so")

MLP_MAX_LAYERS = 4

STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_STATE", 3: "LBM_ERR_OOM", 4: "LBM_ERR_CUDA",
          5: "LBM_ERR_NONFINITE", 6: "LBM_ERR_TIMEOUT", 7: "LBM_ERR_UNSUPPORTED"}


class LbmAllocator(Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, c_void_p, c_void_p)),
                ("ctx", c_void_p)]


class LbmConfig(Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("tau", c_double), ("collision", c_int32),
                ("mrt_rates", c_double * 9), ("precision", c_int32), ("x_periodic", c_int32),
                ("u_in", c_double), ("v_pert_amp", c_double), ("seed", c_uint64),
                ("rho_out", c_double), ("stream", c_void_p), ("alloc", POINTER(LbmAllocator)),
                ("force_capacity", c_int64), ("ramp_steps", c_int64), ("layout", c_int32)]


class LbmMlp(Structure):
    _fields_ = [("n_layers", c_int32), ("sizes", c_int32 * (MLP_MAX_LAYERS + 1)), ("act", c_int32),
                ("params", POINTER(c_float)), ("n_params", c_int64), ("in_mean", POINTER(c_float)),
                ("in_std", POINTER(c_float)), ("out_scale", c_float)]


class LbmTrainOpts(Structure):
    _fields_ = [("batch_rows", c_int32), ("lr", c_double), ("beta1", c_double),
                ("beta2", c_double), ("eps", c_double), ("adam_t0", c_int64),
                ("max_cluster", c_int32), ("stream", c_void_p)]


class LbmCbcSegments(Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("n_t", c_int32), ("tau", c_double),
                ("rho_out", c_double), ("sigma", c_double), ("kappa2", c_double),
                ("mach", c_double), ("length", c_double), ("exact_mass", c_int32),
                ("precision", c_int32), ("bank", c_void_p), ("n_states", c_int32), ("bank_width", c_int32),
                ("init_state", POINTER(c_int32)), ("final_state", POINTER(c_int32)),
                ("n_seg", c_int32), ("stream", c_void_p)]


# name -> (restype, argtypes); every function of include/lbm.h
SIGNATURES = {
    "lbm_config_default": (c_int, [POINTER(LbmConfig)]),
    "lbm_create": (c_int, [POINTER(LbmConfig), POINTER(c_void_p)]),
    "lbm_destroy": (c_int, [c_void_p]),
    "lbm_set_geometry": (c_int, [c_void_p, POINTER(c_uint8)]),
    "lbm_init_equilibrium": (c_int, [c_void_p, POINTER(c_double), POINTER(c_double),
                                     POINTER(c_double)]),
    "lbm_set_outflow_zouhe": (c_int, [c_void_p, c_double]),
    "lbm_set_outflow_nn": (c_int, [c_void_p, POINTER(LbmMlp), c_double]),
    "lbm_nn_fallbacks": (c_int, [c_void_p, POINTER(c_int64)]),
    "lbm_set_outflow_cbc": (c_int, [c_void_p, c_double, c_double, c_double, c_double,
                                    POINTER(LbmMlp), c_int32]),
    "lbm_capture_plane": (c_int, [c_void_p, c_int32, c_int32, c_void_p, c_int64]),
    "lbm_capture_count": (c_int, [c_void_p, POINTER(c_int64)]),
    "lbm_capture_snapshot": (c_int, [c_void_p, c_int32, c_int32, c_void_p]),
    "lbm_save": (c_int, [c_void_p, c_char_p]),
    "lbm_load": (c_int, [c_void_p, c_char_p]),
    "lbm_nn_dataset_stats": (c_int, [c_void_p, c_int64, c_void_p, POINTER(c_float),
                                     POINTER(c_float), POINTER(c_float)]),
    "lbm_train_opts_default": (c_int, [POINTER(LbmTrainOpts)]),
    "lbm_nn_train": (c_int, [c_void_p, c_int64, POINTER(c_int32), c_int64, POINTER(LbmTrainOpts),
                             POINTER(LbmMlp), POINTER(c_float), POINTER(c_float),
                             POINTER(c_float), POINTER(c_double)]),
    "lbm_nn_loss_grad": (c_int, [c_void_p, c_int64, POINTER(c_int32), c_int64,
                                 POINTER(LbmTrainOpts), POINTER(LbmMlp), POINTER(c_double),
                                 POINTER(c_float)]),
    "lbm_copy_columns": (c_int, [c_void_p, c_int32, c_int32, c_void_p]),
    "lbm_cbc_feature_stats": (c_int, [POINTER(LbmCbcSegments), POINTER(c_float),
                                      POINTER(c_float)]),
    "lbm_cbc_segment_grad": (c_int, [POINTER(LbmCbcSegments), POINTER(LbmMlp), POINTER(c_double),
                                     POINTER(c_double), POINTER(c_double)]),
    "lbm_cbc_tuner_train": (c_int, [POINTER(LbmCbcSegments), POINTER(LbmMlp), POINTER(c_int32),
                                    c_int32, c_int64, POINTER(LbmTrainOpts), POINTER(c_double),
                                    POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
    "lbm_step": (c_int, [c_void_p, c_int64]),
    "lbm_sync": (c_int, [c_void_p]),
    "lbm_time": (c_int, [c_void_p, POINTER(c_int64)]),
    "lbm_forces": (c_int, [c_void_p, POINTER(c_double), POINTER(c_double), c_int64,
                           POINTER(c_int64)]),
    "lbm_fields": (c_int, [c_void_p, POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
    "lbm_get_populations": (c_int, [c_void_p, POINTER(c_double)]),
    "lbm_set_populations": (c_int, [c_void_p, POINTER(c_double)]),
    "lbm_mass": (c_int, [c_void_p, POINTER(c_double)]),
    "lbm_device_state": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_int64), POINTER(c_int64)]),
    "lbm_set_tiling": (c_int, [c_void_p, c_int32, c_int32]),
    "lbm_get_tiling": (c_int, [c_void_p, POINTER(c_int32), POINTER(c_int32)]),
    "lbm_debug_hold_dataflow": (c_int, [c_void_p, c_int32]),
    "lbm_autotune": (c_int, [c_void_p, c_int32, c_int64, POINTER(c_float)]),
    "lbm_step_noalloc": (c_int, [POINTER(LbmConfig), c_void_p, c_void_p, c_void_p, c_int64,
                                 c_int64, c_void_p]),
    "lbm_batch_create": (c_int, [POINTER(c_void_p), c_int32, POINTER(c_void_p)]),
    "lbm_batch_destroy": (c_int, [c_void_p]),
    "lbm_batch_step": (c_int, [c_void_p, c_int64]),
    "lbm_batch_sync": (c_int, [c_void_p]),
    "lbm_batch_set_tiling": (c_int, [c_void_p, c_int32, c_int32]),
    "lbm_batch_get_tiling": (c_int, [c_void_p, POINTER(c_int32), POINTER(c_int32)]),
    "lbm_batch_autotune": (c_int, [c_void_p, c_int32, c_int64, POINTER(c_float)]),
    "lbm_strouhal": (c_int, [POINTER(c_double), c_int64, c_double, c_double, POINTER(c_double)]),
    "lbm_set_default_allocator": (c_int, [POINTER(LbmAllocator)]),
    "lbm_last_error": (c_char_p, []),
    "lbm_version": (c_char_p, []),
}

_lib = None


def load():
    """Load the shared library once and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    # device memory from torch's caching allocator (LBM_TORCH_ALLOCATOR=0: cudaMalloc)
    from . import _torch_alloc
    _torch_alloc.install_default(lib, LbmAllocator)
    return lib
