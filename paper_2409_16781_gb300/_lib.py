"""ctypes declarations of liblbgb.so (the C ABI in include/lbgb.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback for any operation of this package.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbgb.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_EDIVERGED, LB_ETIMEOUT, LB_EBUSY = 0, -1, -2, -3, -4, -5, -6
LB_F64, LB_F32, LB_F16S, LB_BF16S, LB_F32D, LB_E3M12S = 0, 1, 2, 3, 4, 5
STORAGE = {"f64": LB_F64, "f32": LB_F32, "f16s": LB_F16S, "bf16s": LB_BF16S, "f32d": LB_F32D,
           "e3m12s": LB_E3M12S}
STORAGE_BYTES = {LB_F64: 8, LB_F32: 4, LB_F16S: 2, LB_BF16S: 2, LB_F32D: 4, LB_E3M12S: 2}
Q = 19


class LbOptions(ctypes.Structure):
    _fields_ = [
        ("storage", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("block", ctypes.c_int),
        ("rounding", ctypes.c_int),
        ("force", ctypes.c_double * 3),
        ("stream", ctypes.c_void_p),
        ("trt_magic", ctypes.c_double),
        ("inplace", ctypes.c_int),
        ("halo_z", ctypes.c_int),
        ("reserved", ctypes.c_int * 4),
    ]


class LbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


class LbDiverged(LbError):
    pass


_lib = None
# every exported name and its (restype, argtypes)
_P, _I, _D, _S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_I64 = ctypes.c_int64
SIGNATURES = {
    "lb_default_options": (None, [_P]),
    "lb_velocity_set": (_I, [_P, _P]),
    "lb_bytes_required": (_S, [_I, _I, _I, _P]),
    "lb_create": (_I, [_P, _I, _I, _I, _D, _P, _P, _P]),
    "lb_create_in": (_I, [_P, _I, _I, _I, _D, _P, _P, _P, _P, _S]),
    "lb_init_fields": (_I, [_P, _P, _P]),
    "lb_step": (_I, [_P, _I]),
    "lb_moments": (_I, [_P, _P, _P]),
    "lb_moments_device": (_I, [_P, _P, _P]),
    "lb_totals": (_I, [_P, _P, _P]),
    "lb_get_populations": (_I, [_P, _P]),
    "lb_set_populations": (_I, [_P, _P]),
    "lb_get_populations_at": (_I, [_P, _P, _I, _P]),
    "lb_checkpoint_bytes": (_S, [_P]),
    "lb_checkpoint_save": (_I, [_P, _P, _S]),
    "lb_checkpoint_load": (_I, [_P, _P, _S]),
    "lb_set_kernel": (_I, [_P, _I, _I]),
    "lb_autotune": (_I, [_P, _I, _P, _P, _P]),
    "lb_totals_static": (_I, [_P, _I64, _P, _I, _I, _I, _I, _P, _P, _P, _P]),
    "lb_batch_slot_bytes": (_S, [_I, _I, _I, _I, _I]),
    "lb_batch_fixed_bytes": (_S, [_I]),
    "lb_batch_create": (_I, [_P, _S, _I, _P]),
    "lb_batch_create_in": (_I, [_P, _P, _S, _I, _P]),
    "lb_batch_add": (_I, [_P, _I, _I, _I, _D, _P, _P, _P, _I64, _P]),
    "lb_batch_set_steps": (_I, [_P, _I, _I64]),
    "lb_batch_set_steps_many": (_I, [_P, _I, _P, _P]),
    "lb_batch_init_fields": (_I, [_P, _I, _P, _P]),
    "lb_batch_step": (_I, [_P, _I]),
    "lb_batch_poll": (_I, [_P, _P, _I, _P]),
    "lb_batch_query": (_I, [_P, _I, _P, _P, _P, _P]),
    "lb_batch_moments": (_I, [_P, _I, _P, _P]),
    "lb_batch_totals": (_I, [_P, _I, _P, _P]),
    "lb_batch_get_populations": (_I, [_P, _I, _P]),
    "lb_batch_fetch": (_I, [_P, _I, _P, _P]),
    "lb_batch_fetch_done": (_I, [_P, _I]),
    "lb_batch_remove": (_I, [_P, _I]),
    "lb_batch_free_bytes": (_I, [_P, _P, _P]),
    "lb_batch_sync": (_I, [_P]),
    "lb_batch_destroy": (_I, [_P]),
    "lb_batch_last_error": (ctypes.c_char_p, []),
    "lb_halo_bytes": (_S, [_P]),
    "lb_halo_pack": (_I, [_P, _P, _P]),
    "lb_halo_unpack": (_I, [_P, _P, _P]),
    "lb_selftest_wait": (_I, [_D, _P]),
    "lb_sync": (_I, [_P]),
    "lb_query": (_I, [_P, _P, _P, _P]),
    "lb_destroy": (_I, [_P]),
    "lb_status_string": (ctypes.c_char_p, [_I]),
    "lb_last_error": (ctypes.c_char_p, []),
}


def lib():
    """The loaded liblbgb.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"liblbgb.so not found at {LIB_PATH}: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def load(path: str):
    """Another build of the library (the bounds-checked test build), with the
    same signatures; loaded RTLD_LOCAL beside liblbgb.so."""
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def check(status: int, what: str = "") -> int:
    if status == LB_OK:
        return status
    L = lib()
    msg = L.lb_last_error().decode() or L.lb_status_string(status).decode()
    cls = LbDiverged if status == LB_EDIVERGED else LbError
    raise cls(status, f"{what}: {msg}" if what else msg)
