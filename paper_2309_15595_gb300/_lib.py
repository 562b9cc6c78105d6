"""ctypes binding of the C ABI declared in include/chase.h.

Argument marshalling only: every step of the eigensolver runs in the CUDA
kernels of ``libchase_gb300.so``. Importing this module loads the in-tree
library and raises if it has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchase_gb300.so")

CHASE_OK = 0
CHASE_ERR_INVALID_ARG = 1
CHASE_ERR_CUDA = 2
CHASE_ERR_OOM = 3
CHASE_ERR_QR_BREAKDOWN = 4
CHASE_ERR_HEEV_NOCONV = 5
CHASE_ERR_NOT_CONVERGED = 6

CHASE_FP64 = 0
CHASE_MIXED_BF16X3 = 1

CHASE_QR_CHOLQR1 = 1
CHASE_QR_CHOLQR2 = 2
CHASE_QR_SHIFTED = 3
CHASE_QR_HOUSEHOLDER = 4
CHASE_QR_FALLBACK = CHASE_QR_HOUSEHOLDER  # former name


class ChaseParams(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64), ("nev", ctypes.c_int64), ("nex", ctypes.c_int64),
        ("deg_init", ctypes.c_int32), ("deg_max", ctypes.c_int32),
        ("deg_extra", ctypes.c_int32), ("deg_opt", ctypes.c_int32),
        ("max_iter", ctypes.c_int32), ("lanczos_steps", ctypes.c_int32),
        ("lanczos_vecs", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("scaled_filter", ctypes.c_int32), ("fp64_tensor", ctypes.c_int32),
        ("tol", ctypes.c_double), ("switch_tol", ctypes.c_double),
        ("heev_max_sweeps", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class ChaseStats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32), ("locked", ctypes.c_int32),
        ("matvecs", ctypes.c_int64), ("matvecs_mixed", ctypes.c_int64),
        ("b_sup", ctypes.c_double), ("mu_1", ctypes.c_double),
        ("mu_ne", ctypes.c_double), ("norm_est", ctypes.c_double),
        ("ms_lanczos", ctypes.c_double), ("ms_filter", ctypes.c_double),
        ("ms_qr", ctypes.c_double), ("ms_rr", ctypes.c_double),
        ("ms_resid", ctypes.c_double), ("ms_total", ctypes.c_double),
        ("filter_flops", ctypes.c_double),
        ("qr_variant_count", ctypes.c_int32 * 5),
        ("switch_iter", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int64),
        ("heev_sweeps", ctypes.c_int32), ("heev_fp64_sweeps", ctypes.c_int32),
        ("ms_heev", ctypes.c_double),
        ("heev_cluster_solves", ctypes.c_int32), ("heev_cluster_max", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["qr_variant_count"] = list(self.qr_variant_count)
        return d


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double

# name: (restype, argtypes); every symbol include/chase.h declares
SIGNATURES = {
    "chase_default_params": (None, [ctypes.POINTER(ChaseParams), _i64, _i64, _i64]),
    "chase_create": (ctypes.c_int, [ctypes.POINTER(ChaseParams), _vp, ctypes.POINTER(_vp)]),
    "chase_destroy": (ctypes.c_int, [_vp]),
    "chase_solve": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _vp,
                                   ctypes.POINTER(ChaseStats)]),
    "chase_lanczos": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _i64, ctypes.POINTER(_dbl)]),
    "chase_filter": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _i64, ctypes.POINTER(_i32),
                                    _dbl, _dbl, _dbl, _i32]),
    "chase_qr": (ctypes.c_int, [_vp, _vp, _i64, _i64, _dbl, ctypes.POINTER(_i32)]),
    "chase_rayleigh_ritz": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _i64, _vp]),
    "chase_residuals": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp]),
    "chase_residuals_noalloc": (ctypes.c_int, [_vp, _i64, _vp, _i64, _vp, _i64, _i64, _vp, _vp]),
    "chase_solve_batch": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                         ctypes.POINTER(ChaseStats), ctypes.POINTER(_i32), _i32]),
    "chase_filter_vjp": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _i64, _i32, _dbl, _dbl, _dbl,
                                        _vp, _i64, _vp, _i64, _vp, _i64, _i32]),
    "chase_eig_vjp": (ctypes.c_int, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _i64, _vp, _vp, _i64,
                                     _vp, _i64, _dbl, _i32, ctypes.POINTER(_i32)]),
    "chase_cond_est": (_dbl, [ctypes.POINTER(_dbl), ctypes.POINTER(_i32), _i64, _i64, _dbl, _dbl]),
    "chase_degree_opt": (None, [ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), _i64, _dbl, _dbl, _dbl,
                                _i32, _i32, ctypes.POINTER(_i32)]),
    "chase_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = load()
