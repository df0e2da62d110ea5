"""ctypes view of the C ABI in include/spl.h (no torch here).

The shared library is the in-tree build paper_2004_09211_gb300/lib/libspl.so. Loading fails loudly when it
is missing: there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libspl.so")

SPL_OK, SPL_EINVAL, SPL_ENOMEM, SPL_ECUDA, SPL_ETIMEOUT, SPL_EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "SPL_OK", 1: "SPL_EINVAL", 2: "SPL_ENOMEM", 3: "SPL_ECUDA", 4: "SPL_ETIMEOUT",
                5: "SPL_EUNSUPPORTED"}
SPL_HIST_U16, SPL_HIST_F16, SPL_HIST_F32 = 0, 1, 2
SPL_MAX_TAPS = 128
SPL_MAX_BINS = 8192
SPL_MAX_BANDS = 8


class spl_params(ct.Structure):
    _fields_ = [("H", ct.c_int32), ("W", ct.c_int32), ("T", ct.c_int32), ("L", ct.c_int32),
                ("peak", ct.c_int32), ("dmin", ct.c_int32), ("dmax", ct.c_int32), ("beta", ct.c_float),
                ("sigma_rw2", ct.c_float), ("nu", ct.c_float * 9)]


class spl_hist(ct.Structure):
    _fields_ = [("fmt", ct.c_int), ("data", ct.c_void_p), ("pitch", ct.c_int64)]


class spl_seq_frame(ct.Structure):
    _fields_ = [(n, ct.c_void_p) for n in ("h", "offsets", "bins", "mu_in", "var_in", "present_in", "faulty",
                                           "present_now", "mu_out", "var_out", "argmax", "refl", "bg")]


class spl_seq_desc(ct.Structure):
    _fields_ = [("prm", spl_params), ("f", spl_seq_frame)]


SPL_NOALLOC_MAX_SEQ = 4096
SPL_BATCH_BAD_BIN = 1
SPL_BATCH_TOO_MANY = 2
SPL_BATCH_DESC_MISMATCH = 4
SPL_MAX_PHOTONS = 1024
SPL_TOA_BAD_BIN = 1
SPL_TOA_SATURATED = 2
SPL_TOA_BAD_OFFSETS = 4


# name -> (restype, argtypes); mirrors include/spl.h
_P = ct.POINTER(spl_params)
_Hh = ct.POINTER(spl_hist)
_vp = ct.c_void_p
SIGNATURES = {
    "spl_version": (ct.c_char_p, []),
    "spl_last_error": (ct.c_char_p, []),
    "spl_probe_throughput": (ct.c_int, [ct.c_int, ct.c_int, ct.c_int, _vp, _vp, ct.POINTER(ct.c_int),
                                        ct.POINTER(ct.c_longlong), _vp]),
    "spl_depth_cost": (ct.c_int, [_P, _Hh, _vp, _vp, _vp, _vp]),
    "spl_depth_cost_tc": (ct.c_int, [_P, _Hh, _vp, _vp, _vp, _vp]),
    "spl_tc_status": (ct.c_int, [ct.POINTER(ct.c_uint32)]),
    "spl_depth_estimate": (ct.c_int, [_P, _Hh, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "spl_filter_step": (ct.c_int, [_P, _Hh, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "spl_depth_estimate_fine": (ct.c_int, [_P, ct.c_int, _Hh, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "spl_depth_estimate_msl": (ct.c_int, [_P, ct.c_int, _Hh, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "spl_filter_step_detect": (ct.c_int, [_P, _Hh, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                          _vp, _vp]),
    "spl_filter_step_tc": (ct.c_int, [_P, _Hh, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "spl_filter_step_fp32": (ct.c_int, [_P, _Hh, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "spl_state_init": (ct.c_int, [_P, _vp, _vp, _vp]),
    "spl_pi_propagate": (ct.c_int, [_P, _vp, _vp, _vp, _vp]),
    "spl_batch_create": (ct.c_int, [_P, ct.c_int, ct.c_int, ct.POINTER(ct.c_void_p)]),
    "spl_batch_destroy": (None, [_vp]),
    "spl_batch_set": (ct.c_int, [_vp, ct.c_int, ct.POINTER(spl_seq_frame)]),
    "spl_batch_step": (ct.c_int, [_vp, ct.c_int, _vp]),
    "spl_batch_tune": (ct.c_int, [_vp, ct.c_int, _vp]),
    "spl_batch_info": (ct.c_int, [_vp] + [ct.POINTER(ct.c_int)] * 4),
    "spl_batch_class_info": (ct.c_int, [_vp, ct.c_int] + [ct.POINTER(ct.c_int)] * 5),
    "spl_batch_status": (ct.c_int, [_vp, ct.POINTER(ct.c_uint32)]),
    "spl_diff_scratch_size": (ct.c_int, [_P, ct.POINTER(ct.c_size_t)]),
    "spl_diff_forward": (ct.c_int, [_P, ct.c_int, _Hh, _vp, ct.c_float, _vp, _vp, _vp, _vp, _vp, _vp, ct.c_size_t, _vp]),
    "spl_diff_backward": (ct.c_int, [_P, ct.c_int, _Hh, _vp, ct.c_float, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ct.c_size_t,
                                     _vp]),
    "spl_toa_histogram": (ct.c_int, [_P, _vp, _vp, ct.c_int64, _vp, ct.c_int64, _vp]),
    "spl_toa_status": (ct.c_int, [ct.POINTER(ct.c_uint32)]),
    "spl_batch_step_noalloc": (ct.c_int, [ct.POINTER(spl_seq_desc), _vp, ct.c_int, ct.c_int, _vp, _vp]),
}

_lock = threading.Lock()
_lib = None


class SplError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def load(path: str | None = None) -> ct.CDLL:
    """Load libspl.so (building it first if the sources are newer). Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if path is None:
                from . import build as _build
                if not _build.up_to_date():
                    _build.build()
            if not os.path.exists(p):
                raise RuntimeError(f"libspl.so not found at {p}; build it with paper_2004_09211_gb300.build")
            lib = ct.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int) -> None:
    if status != SPL_OK:
        msg = load().spl_last_error()
        raise SplError(status, msg.decode() if msg else "")
