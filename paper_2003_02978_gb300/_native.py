"""ctypes declarations of libmf.so (the C ABI of include/mf.h)."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_uint32, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmf.so")

MF_OK = 0
STATUS_NAMES = {0: "MF_OK", 1: "MF_ERR_INVALID_ARG", 2: "MF_ERR_CUDA", 3: "MF_ERR_OOM",
                4: "MF_ERR_NOT_SPD", 5: "MF_ERR_NONFINITE_INPUT", 6: "MF_ERR_TIMEOUT",
                7: "MF_ERR_INTERNAL", 8: "MF_ERR_UNSUPPORTED"}


class MfTuning(ctypes.Structure):
    _fields_ = [("pixel_rows", c_int32), ("stat_rows", c_int32), ("use_graph", c_int32)]


class MfDesc(ctypes.Structure):
    _fields_ = [("rows", c_int64), ("cols", c_int64), ("bands_total", c_int64),
                ("band_lo", c_int32), ("band_hi", c_int32), ("col_group", c_int32),
                ("layout", c_int32), ("precision", c_int32), ("flags", c_uint32)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libmf.so; fails loudly when it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2003_02978_gb300.build` "
            "(the CUDA path has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    fp = c_void_p
    L.mf_plan.argtypes = [POINTER(MfDesc), POINTER(c_void_p)]
    L.mf_plan.restype = c_int
    L.mf_destroy.argtypes = [c_void_p]
    L.mf_destroy.restype = None
    L.mf_num_partitions.argtypes = [c_void_p]
    L.mf_num_partitions.restype = c_int64
    L.mf_retrieve.argtypes = [c_void_p, fp, fp, c_double, c_double, c_int32, fp, fp, fp, fp,
                              c_void_p]
    L.mf_retrieve.restype = c_int
    L.mf_retrieve_host.argtypes = [c_void_p, fp, fp, c_double, c_double, c_int32, fp, fp,
                                   c_void_p]
    L.mf_retrieve_host.restype = c_int
    L.mf_retrieve_host_async.argtypes = [c_void_p, fp, fp, c_double, c_double, c_int32, fp, fp,
                                         c_void_p]
    L.mf_retrieve_host_async.restype = c_int
    L.mf_background.argtypes = [c_void_p, fp, fp, c_void_p]
    L.mf_background.restype = c_int
    L.mf_plan_status.argtypes = [c_void_p, POINTER(c_int32)]
    L.mf_plan_status.restype = c_int
    L.mf_status_string.argtypes = [c_int]
    L.mf_status_string.restype = c_char_p
    L.mf_last_error.argtypes = []
    L.mf_last_error.restype = c_char_p
    L.mf_background_noalloc.argtypes = [POINTER(MfDesc), fp, fp, fp, fp, c_void_p]
    L.mf_background_noalloc.restype = c_int
    L.mf_plan_batched.argtypes = [POINTER(MfDesc), POINTER(c_int64), c_int32, POINTER(c_void_p)]
    L.mf_plan_batched.restype = c_int
    L.mf_plan_ex.argtypes = [POINTER(MfDesc), POINTER(c_int64), c_int32, POINTER(MfTuning),
                             POINTER(c_void_p)]
    L.mf_plan_ex.restype = c_int
    L.mf_ckpt_bytes.argtypes = [c_void_p, c_int32, c_int32]
    L.mf_ckpt_bytes.restype = ctypes.c_size_t
    L.mf_retrieve_train.argtypes = [c_void_p, fp, fp, c_double, c_double, c_int32, fp, fp, fp,
                                    c_int32, c_void_p]
    L.mf_retrieve_train.restype = c_int
    L.mf_retrieve_backward.argtypes = [c_void_p, fp, fp, fp, fp, fp, c_void_p]
    L.mf_retrieve_backward.restype = c_int
    L.mf_num_lines.argtypes = [c_void_p]
    L.mf_num_lines.restype = c_int32
    L.mf_retrieve_energy.argtypes = [c_void_p, fp, fp, c_double, c_double, c_int32, fp, fp, fp,
                                     c_void_p]
    L.mf_retrieve_energy.restype = c_int
    L.mf_retrieve_batched.argtypes = [c_void_p, fp, fp, POINTER(c_double), c_double,
                                      POINTER(c_int32), fp, fp, c_void_p]
    L.mf_retrieve_batched.restype = c_int
    for name, args in (("mf_profile", [c_void_p, c_int32]),
                       ("mf_profile_read", [c_void_p, POINTER(c_double), POINTER(c_int64),
                                            c_int32]),
                       ("mf_timeline", [c_void_p, c_int32]),
                       ("mf_timeline_read", [c_void_p, POINTER(c_double), POINTER(c_double),
                                             POINTER(c_int32), c_int32, POINTER(c_int32)])):
        if hasattr(L, name):
            getattr(L, name).argtypes = args
            getattr(L, name).restype = c_int
    _lib = L
    return L


class MFError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().mf_last_error().decode() if _lib is not None else ""
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {msg}".strip())
        self.status = status


def check(status: int, where: str) -> None:
    if status != MF_OK:
        raise MFError(status, where)
