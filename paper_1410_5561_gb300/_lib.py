"""ctypes binding of the C ABI in include/stencil_gb300.h (argument marshalling only).

Loading fails loudly when ``libstencil_gb300.so`` has not been built: there is
no CPU fallback for any operation of this library.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstencil_gb300.so")

STENCIL_7PT_CONST, STENCIL_7PT_VAR, STENCIL_25PT_VAR = 0, 1, 2
STENCIL_F32, STENCIL_F64, STENCIL_BF16 = 0, 1, 2
STENCIL_PLAIN, STENCIL_BLOCKED, STENCIL_AUTO, STENCIL_WAVEFRONT = 0, 1, 2, 3
STENCIL_HOST, STENCIL_DEVICE, STENCIL_HOST_ASYNC = 0, 1, 2
STENCIL_FIELD_ARRAY, STENCIL_COEF_ARRAY, STENCIL_GRAD_ARRAY = 0, 1, 2

STATUS = {0: "STENCIL_OK", -1: "STENCIL_EINVAL", -2: "STENCIL_ENOSMEM", -3: "STENCIL_ETIMEOUT",
          -4: "STENCIL_ECUDA", -5: "STENCIL_EUNBOUND", -6: "STENCIL_ENOTSUP"}


class stencil_tuning(ctypes.Structure):
    _fields_ = [("dw", ctypes.c_int), ("nf", ctypes.c_int), ("warps", ctypes.c_int),
                ("xtile", ctypes.c_int)]


class stencil_layout(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_int), ("elem_bytes", ctypes.c_int), ("x_offset", ctypes.c_int),
                ("pitch_x", ctypes.c_int), ("pitch_y", ctypes.c_int), ("planes", ctypes.c_int),
                ("bytes", ctypes.c_size_t)]


class StencilError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn} failed: {STATUS.get(status, status)} "
                         f"({lib().stencil_strerror(status).decode()})")


_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every exported entry point declared in the header.
_H = ctypes.c_void_p
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = [
    ("stencil_create", _I, [ctypes.POINTER(_H), _I, _I, _I, _I, _I, _I, _P]),
    ("stencil_layout_of", _I, [_H, _I, ctypes.POINTER(stencil_layout)]),
    ("stencil_workspace_bytes", ctypes.c_size_t, [_H]),
    ("stencil_bind", _I, [_H, _P, _P, ctypes.POINTER(_P), _P]),
    ("stencil_set_coeffs", _I, [_H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_P), _I]),
    ("stencil_set_field", _I, [_H, _P, ctypes.c_double, _I]),
    ("stencil_set_tuning", _I, [_H, _I, ctypes.POINTER(stencil_tuning)]),
    ("stencil_run", _I, [_H, _I]),
    ("stencil_parity", _I, [_H]),
    ("stencil_get_field", _I, [_H, _P, _I]),
    ("stencil_blocked_smem_bytes", ctypes.c_size_t, [_H, ctypes.POINTER(stencil_tuning)]),
    ("stencil_launch_count", _I, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    ("stencil_tile_copy_passes", _I, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    ("stencil_copy", _I, [_P, _P, ctypes.c_size_t, _I, _P]),
    ("stencil_adjoint_workspace_bytes", ctypes.c_size_t, [_H, _I, _I]),
    ("stencil_run_checkpointed", _I, [_H, _I, _I, _P, ctypes.c_size_t]),
    ("stencil_run_adjoint", _I, [_H, _I, _I, _P, _P, ctypes.POINTER(_P), _P, ctypes.c_size_t]),
    ("stencil_probe_fma", _I, [_I, _I, _P, _P, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]),
    ("stencil_batch_create", _I, [ctypes.POINTER(_H), ctypes.POINTER(_H), ctypes.POINTER(_I), _I,
                                  ctypes.POINTER(stencil_tuning)]),
    ("stencil_batch_workspace_bytes", ctypes.c_size_t, [_H]),
    ("stencil_batch_item_count", _I, [_H]),
    ("stencil_batch_bind", _I, [_H, _P, _P]),
    ("stencil_batch_launch", _I, [_H, _P]),
    ("stencil_batch_launch_count", _I, [_H, ctypes.POINTER(ctypes.c_longlong)]),
    ("stencil_batch_status", _I, [_H, ctypes.POINTER(_I)]),
    ("stencil_batch_sync_parity", _I, [_H]),
    ("stencil_batch_set_wait_limit", _I, [_H, ctypes.c_uint]),
    ("stencil_batch_inject_stall", _I, [_H, _I]),
    ("stencil_batch_destroy", _I, [_H]),
    ("stencil_batch_run_noalloc", _I, [ctypes.POINTER(_H), ctypes.POINTER(_I), _I, ctypes.POINTER(stencil_tuning),
                                       _P, ctypes.POINTER(_I)]),
    ("stencil_set_stream", _I, [_H, _P]),
    ("stencil_sync", _I, [_H]),
    ("stencil_status", _I, [_H]),
    ("stencil_set_wait_limit", _I, [_H, ctypes.c_uint]),
    ("stencil_inject_stall", _I, [_H, _I]),
    ("stencil_strerror", ctypes.c_char_p, [_I]),
    ("stencil_destroy", _I, [_H]),
]


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(fn: str, status: int) -> int:
    if status < 0:
        raise StencilError(fn, status)
    return status


def call(name: str, *args):
    """Call entry point ``name``; raise StencilError on a negative status."""
    f = getattr(lib(), name)
    r = f(*args)
    if f.restype is _I:
        check(name, r)
    return r
