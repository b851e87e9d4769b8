"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

The shared library is ``paper_1710_09472_gb300/_build/liblbm.so``, built in
tree by ``paper_1710_09472_gb300.build.build()``.  There is no fallback: if
the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")

LBM_OK = 0
STATUS = {0: "LBM_OK", 1: "LBM_ERR_INVALID_ARG", 2: "LBM_ERR_UNSTABLE_LATTICE", 3: "LBM_ERR_CUDA", 4: "LBM_ERR_OOM",
          5: "LBM_ERR_NONFINITE", 6: "LBM_ERR_TIMEOUT", 7: "LBM_ERR_STATE"}
VEL = {"D2V9": 0, "D3V19": 1, "D3V27": 2, "D1V3": 3}
STAT = {"fd": 0, "be": 1, "mb": 2}
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
FORCE = {"shift": 0, "term": 1}

# Every symbol include/lbm.h declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_d = ctypes.c_double
_i = ctypes.c_int
SIGNATURES = {
    "lbm_create": (_i, [ctypes.POINTER(_vp), _vp, _vp, _d, _vp, _vp, _i, _vp]),
    "lbm_destroy": (None, [_vp]),
    "lbm_constants": (_i, [_vp, _vp, _i]),
    "lbm_info": (_i, [_vp, _vp, _i]),
    "lbm_set_geometry": (_i, [_vp, _vp]),
    "lbm_set_E_field": (_i, [_vp, _vp]),
    "lbm_set_params": (_i, [_vp, _d, _vp, _vp]),
    "lbm_set_rounding": (_i, [_vp, _i]),
    "lbm_set_rounding_seed": (_i, [_vp, ctypes.c_uint32]),
    "lbm_set_local_mu": (_i, [_vp, _i]),
    "lbm_thermal_create": (_i, [ctypes.POINTER(_vp), _i, _i, _d, _d, _i64, _d, _d, _i, _i, _vp]),
    "lbm_thermal_destroy": (None, [_vp]),
    "lbm_thermal_constants": (_i, [_vp, _vp, _i]),
    "lbm_thermal_set_rounding": (_i, [_vp, _i, ctypes.c_uint32]),
    "lbm_thermal_init": (_i, [_vp, _vp, _vp, _vp]),
    "lbm_thermal_step": (_i, [_vp, _i64]),
    "lbm_thermal_moments": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_thermal_populations": (_i, [_vp, _vp, _i]),
    "lbm_thermal_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_thermal_launch_count": (_i64, [_vp]),
    "lbm_density_from_mu": (_i, [_i, _d, _vp, _vp, _i64, _vp]),
    "lbm_mu_from_density": (_i, [_i, _d, _vp, _vp, _i64, _vp]),
    "lbm_init_equilibrium": (_i, [_vp, _vp, _vp]),
    "lbm_step": (_i, [_vp, _i64]),
    "lbm_moments": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_get_populations": (_i, [_vp, _vp, _i]),
    "lbm_save_state": (_i, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_load_state": (_i, [_vp, _vp, ctypes.c_size_t]),
    "lbm_window_totals": (_i, [_vp, _i64, _i64, _vp]),
    "lbm_adjoint": (_i, [_vp, _vp, _vp, _i64, _i64, _i64, _vp, _vp, _vp, _vp, _vp]),
    "lbm_weight_integrals": (_i, [_i, _i, _d, _d, _vp]),
    "lbm_moment_totals_static": (_i, [_vp, _vp]),
    "lbm_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_status_string": (ctypes.c_char_p, [_i]),
    "lbm_launch_count": (_i64, [_vp]),
    "lbm_selftest_wait_timeout": (_i, [_vp, _i64]),
    "lbm_set_memory_budget": (_i, [_vp, ctypes.c_uint64]),
    "lbm_adjoint_stats": (_i, [_vp, _vp]),
    "lbm_release_workspace": (_i, [_vp]),
}


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class lbm_lattice(ctypes.Structure):
    _fields_ = [("vel", ctypes.c_int), ("stat", ctypes.c_int), ("theta", ctypes.c_double),
                ("mu", ctypes.c_double), ("force", ctypes.c_int), ("rho0", ctypes.c_double)]


_lib = None


def load():
    """Load liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"liblbm.so is not built ({LIB_PATH}); run paper_1710_09472_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


THERMAL_LATTICE = {"D1V5a": 0, "D1V5b": 1, "D1V7": 2, "D1V7r1": 3, "D1V7r2": 4}


def check(status: int, ctx=None, what: str = "", thermal: bool = False):
    if status != LBM_OK:
        msg = ""
        if ctx:
            getter = load().lbm_thermal_last_error if thermal else load().lbm_last_error
            msg = (getter(ctx) or b"").decode()
        raise LBMError(status, f"{what}: {msg}" if what else msg)
