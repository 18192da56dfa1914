"""ctypes loader for the SMART CUDA library (``_lib/libsmart.so``).

There is no fallback: if the library is missing or fails to load, importing
the package's GPU API raises.  Build it with
``python -m paper_2609_11181_b300.build``.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsmart.so")

STATUS = {0: "SMART_OK", 1: "SMART_E_ARG", 2: "SMART_E_NOMEM", 3: "SMART_E_CUDA", 4: "SMART_E_STATE",
          5: "SMART_E_TIMEOUT", 6: "SMART_E_OVERFLOW", 7: "SMART_E_INTERNAL"}

KERNELS = {"pixel_toeplitz": 0, "pixel_general": 1, "galaxy": 2, "galaxy_band": 3, "galaxy_finalise": 4,
           "bin_keys": 5, "bin_sort": 6, "bin_records": 7, "bin_pixel_sums": 8, "bary_build": 9, "bary_map": 10,
           "pixel_band": 11, "proj_records": 12, "proj_map": 13, "proj_band": 14}

MLP_FEATURES = 4
MLP_NPARAMS = 4545
MLP_BF16 = 0
MLP_FP32 = 1

FILTER_POLY = 1
FILTER_SCHIRMER = 2
FILTER_JARVIS = 3


class SmartFilter(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("xc", ctypes.c_double)]


class SmartMaps(ctypes.Structure):
    _fields_ = [("sum_w", ctypes.c_void_p), ("map_e", ctypes.c_void_p), ("map_b", ctypes.c_void_p),
                ("var", ctypes.c_void_p), ("count", ctypes.c_void_p), ("members", ctypes.c_void_p)]


# every symbol declared in include/smart.h, with its ctypes signature
_VP, _I64, _I32, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "smart_create": (_I32, [_I32, ctypes.POINTER(SmartFilter), _D, _I32, _VP, ctypes.POINTER(_VP)]),
    "smart_destroy": (None, [_VP]),
    "smart_sync": (_I32, [_VP, _D]),
    "smart_last_error": (ctypes.c_char_p, [_VP]),
    "smart_set_targets": (_I32, [_VP, _VP, _I64]),
    "smart_bin_galaxies": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, _I64]),
    "smart_set_binned": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "smart_set_binned_packed": (_I32, [_VP, _VP, _VP]),
    "smart_map_bruteforce": (_I32, [_VP, ctypes.POINTER(SmartMaps)]),
    "smart_map_pixel": (_I32, [_VP, ctypes.POINTER(SmartMaps)]),
    "smart_map_barycentre": (_I32, [_VP, ctypes.POINTER(SmartMaps)]),
    "smart_set_normalisation": (_I32, [_VP, _I32]),
    "smart_ang2pix": (_I32, [_I32, _VP, _VP, _I64, _VP, _VP]),
    "smart_pix2vec": (_I32, [_I32, _VP, _I64, _VP, _VP]),
    "smart_chord2": (_D, [_D]),
    "smart_get_catalog": (_I32, [_VP, _VP, _VP, _VP]),
    "smart_get_binned": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "smart_last_fp64_decisions": (_I64, [_VP]),
    "smart_batch_create": (_I32, [ctypes.POINTER(_VP), ctypes.POINTER(SmartMaps), _I32, _I32, _VP, ctypes.POINTER(_VP)]),
    "smart_batch_run": (_I32, [_VP]),
    "smart_batch_info": (_I32, [_VP, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I64),
                                ctypes.POINTER(_D)]),
    "smart_batch_last_error": (ctypes.c_char_p, [_VP]),
    "smart_batch_destroy": (None, [_VP]),
    "smart_map_batched": (_I32, [ctypes.POINTER(_VP), ctypes.POINTER(SmartMaps), _I32]),
    "smart_timing_enable": (_I32, [_VP, _I32]),
    "smart_timing_read": (_I32, [_VP, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_D), _D]),
    "smart_get_general_targets": (_I32, [_VP, _VP, _I64, ctypes.POINTER(_I64)]),
    "smart_get_general_pairs": (_I32, [_VP, _VP, _I64, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "smart_set_band_slot_limit": (_I32, [_VP, _I64]),
    "smart_mlp_features": (_I32, [_VP, ctypes.POINTER(SmartMaps), ctypes.POINTER(SmartMaps), _VP, _VP, _VP, _VP]),
    "smart_mlp_create": (_I32, [_I32, _VP, ctypes.POINTER(_VP)]),
    "smart_mlp_destroy": (None, [_VP]),
    "smart_mlp_last_error": (ctypes.c_char_p, [_VP]),
    "smart_mlp_sync": (_I32, [_VP, _D]),
    "smart_mlp_set_params": (_I32, [_VP, _VP]),
    "smart_mlp_get_params": (_I32, [_VP, _VP]),
    "smart_mlp_set_scaler": (_I32, [_VP, ctypes.POINTER(_D)]),
    "smart_mlp_get_scaler": (_I32, [_VP, ctypes.POINTER(_D)]),
    "smart_mlp_fit_scaler": (_I32, [_VP, _VP, _VP, _VP, _I64]),
    "smart_mlp_gradient": (_I32, [_VP, _VP, _VP, _VP, _I64, _VP]),
    "smart_mlp_train_step": (_I32, [_VP, _VP, _VP, _VP, _I64, ctypes.c_float, _VP]),
    "smart_mlp_step": (_I64, [_VP]),
    "smart_mlp_infer": (_I32, [_VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    "smart_mlp_get_state": (_I32, [_VP, _VP, _I64, ctypes.POINTER(_I64)]),
    "smart_mlp_set_state": (_I32, [_VP, _VP, _I64]),
    "smart_sort_catalog_noalloc": (_I32, [_I32, _VP, _VP, _I64, _VP, _VP, _VP, _VP]),
    "smart_fma_probe": (_I32, [_I32, _I64, _I32, _VP, ctypes.POINTER(_D)]),
    "smart_map_projected": (_I32, [_VP, _D, _D, ctypes.POINTER(SmartMaps)]),
    "smart_set_wait_limit": (_I32, [_VP, _D]),
    "smart_set_binned_runs": (_I32, [_VP, _VP, _VP, _VP, _I64, _I64, _I32]),
    "smart_annulus_stats": (_I32, [_VP, _D, _D, _D, _VP, _VP, _I32, _VP, _VP, _VP]),
}

_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"SMART CUDA library not built: {LIB_PATH} is missing "
                              "(run: python -m paper_2609_11181_b300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class SmartError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
