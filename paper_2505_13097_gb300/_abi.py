"""ctypes binding of the C ABI in include/lbm_stefan.h (argument marshalling only).

Every computation happens in the CUDA library; this module only converts
Python / numpy / torch arguments into pointers and sizes.  If the shared
library is missing the import fails: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "liblbm_stefan.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_NEWTON, LBM_ERR_TIMEOUT, LBM_ERR_STATE = range(6)
LBM_D1Q3, LBM_D2Q9, LBM_D2Q5 = 1, 2, 3
LBM_FP64, LBM_FP32 = 0, 1
LBM_ADIABATIC, LBM_DIRICHLET = 0, 1
LBM_BB_MIRROR, LBM_BB_LINK, LBM_NEU_EQ17 = 0, 1, 2
LBM_IREBM, LBM_EEBM, LBM_ILFBM = 0, 1, 2
LBM_WALL_W, LBM_WALL_E, LBM_WALL_S, LBM_WALL_N = 0, 1, 2, 3
WALLS = {"W": LBM_WALL_W, "E": LBM_WALL_E, "S": LBM_WALL_S, "N": LBM_WALL_N}


class lbm_stefan_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau", ctypes.c_double), ("delta", ctypes.c_double), ("ste", ctypes.c_double),
        ("precision", ctypes.c_int), ("newton_tol", ctypes.c_double),
        ("newton_max_iter", ctypes.c_int), ("bb_mode", ctypes.c_int),
    ]


class lbm_stefan_stats(ctypes.Structure):
    _fields_ = [
        ("energy", ctypes.c_double), ("energy_prev", ctypes.c_double), ("flux", ctypes.c_double),
        ("imbalance", ctypes.c_double), ("imbalance_max", ctypes.c_double),
        ("steps", ctypes.c_longlong), ("newton_nodes", ctypes.c_longlong),
        ("newton_max_iter", ctypes.c_int), ("error", ctypes.c_int),
        ("newton_iters", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class lbm_stefan_problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau", ctypes.c_double), ("delta", ctypes.c_double), ("ste", ctypes.c_double),
        ("wall_kind", ctypes.c_int * 4), ("wall_theta", ctypes.c_double * 4),
    ]


_V = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int
_S = ctypes.c_int   # lbm_status

# name -> (restype, argtypes); the same names as the C functions
SIGNATURES = {
    "lbm_stefan_create": (_S, [ctypes.POINTER(lbm_stefan_params), _V, ctypes.POINTER(_V)]),
    "lbm_stefan_set_bc": (_S, [_V, _I, _I, ctypes.c_double]),
    "lbm_stefan_set_method": (_S, [_V, _I]),
    "lbm_stefan_set_ic": (_S, [_V, _V, _I]),
    "lbm_stefan_step": (_S, [_V, _I]),
    "lbm_stefan_step_timed": (_S, [_V, _I, _D]),
    "lbm_stefan_set_wait_test": (_S, [_V, ctypes.c_double, _I]),
    "lbm_stefan_step_record": (_S, [_V, _I, _V]),
    "lbm_stefan_sync": (_S, [_V]),
    "lbm_stefan_get_fields": (_S, [_V, _V, _V, _V, _I]),
    "lbm_stefan_get_stats": (_S, [_V, ctypes.POINTER(lbm_stefan_stats)]),
    "lbm_stefan_front_position": (_S, [_V, _I, _D, _D, _D, _D]),
    "lbm_stefan_layout": (_S, [_V, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]),
    "lbm_stefan_get_state": (_S, [_V, _V, _I]),
    "lbm_stefan_set_state": (_S, [_V, _V, _I]),
    "lbm_stefan_theta_plane": (_S, [_V, _V]),
    "lbm_stefan_adjoint_seed": (_S, [_V, _V, _V, _V, _D]),
    "lbm_stefan_adjoint_step": (_S, [_V, _V, _V, _V, _V]),
    "lbm_stefan_adjoint_run": (_S, [_V, _I, _V, _V, _V, ctypes.POINTER(ctypes.c_int)]),
    "lbm_stefan_adjoint_finish": (_S, [_V, _V, _V, _I, _D, _D]),
    "lbm_stefan_adjoint_segment": (_S, [_V, _V, _I, _V, _V, _V, ctypes.POINTER(ctypes.c_int)]),
    "lbm_stefan_set_ste": (_S, [_V, ctypes.c_double]),
    "lbm_stefan_destroy": (None, [_V]),
    "lbm_stefan_batch_create": (_S, [_I, ctypes.POINTER(lbm_stefan_problem), _I, ctypes.c_double, _I, _V,
                                     ctypes.POINTER(_V)]),
    "lbm_stefan_batch_set_ic": (_S, [_V, _I, _V, _I]),
    "lbm_stefan_batch_step": (_S, [_V, _I]),
    "lbm_stefan_batch_get_fields": (_S, [_V, _I, _V, _I]),
    "lbm_stefan_batch_get_stats": (_S, [_V, _I, ctypes.POINTER(lbm_stefan_stats)]),
    "lbm_stefan_batch_autotune": (_S, [_V, _I, ctypes.POINTER(ctypes.c_int)]),
    "lbm_stefan_batch_set_schedule": (_S, [_V, _I, _I]),
    "lbm_stefan_batch_destroy": (None, [_V]),
    "lbm_stefan_step_d2q9_noalloc": (_S, [ctypes.POINTER(lbm_stefan_params), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double), _V, _V, _V]),
    "lbm_stefan_last_error": (ctypes.c_char_p, []),
}

_lib = None


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lbm_stefan status %d: %s" % (status, msg))
        self.status = status


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("CUDA library %s is missing: run __graft_entry__.build() "
                              "(there is no CPU fallback)" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def check(status: int):
    if status != LBM_OK:
        raise LBMError(status, load().lbm_stefan_last_error().decode(errors="replace"))
    return status
