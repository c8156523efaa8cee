"""ctypes binding of libgvx (include/gvx.h).  Argument marshalling only: no arithmetic here.

The library is built in-tree by ``paper_2312_02756_gb300.build``; if it is missing or fails to
load, every call raises -- there is no CPU or PyTorch fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

GVX_OK = 0
STATUS_NAMES = {
    0: "GVX_OK", 1: "GVX_ERR_NULL", 2: "GVX_ERR_SIZE", 3: "GVX_ERR_DTYPE", 4: "GVX_ERR_LAYOUT",
    5: "GVX_ERR_ALIGN", 6: "GVX_ERR_OFFSETS", 7: "GVX_ERR_WORKSPACE", 8: "GVX_ERR_CUDA",
    9: "GVX_ERR_TIMEOUT", 10: "GVX_ERR_CAPACITY", 11: "GVX_ERR_ARG",
}
F64, F32 = 0, 1
SOA, AOS = 0, 1
PTETAPHIM, PXPYPZE, PXPYPZM, PTETAPHIE = 0, 1, 2, 3

# Every symbol include/gvx.h declares (the CPU tests check the library exports all of them).
EXPORTS = (
    "gvx_version", "gvx_status_string", "gvx_last_cuda_error",
    "gvx_invariant_mass", "gvx_invariant_mass_bwd",
    "gvx_boost", "gvx_boost_bwd_workspace", "gvx_boost_bwd",
    "gvx_event_pair_masses_workspace", "gvx_event_pair_masses",
    "gvx_event_pair_masses_num_shapes", "gvx_event_pair_masses_shape",
    "gvx_event_pair_masses_get_shape", "gvx_event_pair_masses_set_shape",
    "gvx_event_pair_masses_autotune", "gvx_event_pair_masses_graph_create",
    "gvx_graph_launch", "gvx_graph_destroy", "gvx_device_status",
    "gvx_testing_skip_first_tile", "gvx_event_pair_masses_noalloc",
    "gvx_event_pair_masses_bwd_workspace", "gvx_event_pair_masses_bwd", "gvx_event_pair_select",
    "gvx_invariant_mass_cart", "gvx_lorentz_apply", "gvx_to_pxpypze",
)


class GvxError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        name = STATUS_NAMES.get(status, str(status))
        msg = "%s returned %s" % (where, name) if where else name
        if status == 8 and _lib is not None:
            msg += " (cudaError %d)" % _lib.gvx_last_cuda_error()
        super().__init__(msg)


class LV(ctypes.Structure):
    _fields_ = [("c", ctypes.c_void_p * 4), ("layout", ctypes.c_int32)]


_lib = None
P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int32
SZ = ctypes.c_size_t
LVP = ctypes.POINTER(LV)


def _sigs(lib):
    S = ctypes.c_int32  # gvx_status
    table = {
        "gvx_version": ([], ctypes.c_char_p),
        "gvx_status_string": ([I32], ctypes.c_char_p),
        "gvx_last_cuda_error": ([], I32),
        "gvx_invariant_mass": ([LVP, LVP, P, I64, I32, P], S),
        "gvx_invariant_mass_bwd": ([LVP, LVP, P, P, LVP, LVP, I64, I32, P], S),
        "gvx_boost": ([LVP, LVP, I64, LVP, I64, I32, P], S),
        "gvx_boost_bwd_workspace": ([I64, I64, I32], SZ),
        "gvx_boost_bwd": ([LVP, LVP, I64, LVP, LVP, LVP, I64, I32, P, SZ, P], S),
        "gvx_event_pair_masses_workspace": ([I64], SZ),
        "gvx_event_pair_masses": ([LVP, P, I64, I64, P, P, I64, LVP, P, SZ, P], S),
        "gvx_event_pair_masses_num_shapes": ([], I32),
        "gvx_event_pair_masses_shape": ([I32, ctypes.POINTER(I32), ctypes.POINTER(I32)], S),
        "gvx_event_pair_masses_get_shape": ([I64], I32),
        "gvx_event_pair_masses_set_shape": ([I64, I32], S),
        "gvx_event_pair_masses_autotune": ([LVP, P, I64, I64, P, P, I64, LVP, P, SZ, I32, P,
                                            ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_float)],
                                           S),
        "gvx_event_pair_masses_graph_create": ([LVP, P, I64, I64, P, P, I64, LVP, P, SZ,
                                                ctypes.POINTER(P)], S),
        "gvx_graph_launch": ([P, P], S),
        "gvx_graph_destroy": ([P], S),
        "gvx_device_status": ([P, ctypes.POINTER(I32)], S),
        "gvx_testing_skip_first_tile": ([I32], None),
        "gvx_event_pair_masses_noalloc": ([LVP, P, I64, I64, P, P, I64, LVP, P], S),
        "gvx_event_pair_masses_bwd_workspace": ([I64], SZ),
        "gvx_event_pair_masses_bwd": ([LVP, P, P, I64, I64, P, I64, LVP, LVP, P, SZ, P], S),
        "gvx_invariant_mass_cart": ([LVP, LVP, P, I64, I32, I32, P], S),
        "gvx_lorentz_apply": ([P, I64, LVP, LVP, I64, I32, P], S),
        "gvx_to_pxpypze": ([LVP, LVP, I64, I32, I32, P], S),
        "gvx_event_pair_select": ([LVP, P, I64, I64, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, I32, ctypes.c_double, P, P,
                                   P, P], S),
    }
    for name, (args, res) in table.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libgvx (building it first if it is missing or stale and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libgvx is not built (%s); run paper_2312_02756_gb300.build" % path)
    lib = ctypes.CDLL(path)
    _sigs(lib)
    _lib = lib
    return lib


def check(status, where=""):
    if status != GVX_OK:
        raise GvxError(status, where)
