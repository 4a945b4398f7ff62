"""ctypes binding of ``libpip.so`` (declared in ``include/pip.h``).

Argument marshalling only: every function here forwards raw device pointers and sizes to the
C ABI of the same name.  Loading fails loudly when the library has not been built; there is
no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpip.so")

PIP_OK = 0
PIP_ERR_NULL = -1
PIP_ERR_SIZE = -2
PIP_ERR_ALIGN = -3
PIP_ERR_TOO_LARGE = -4
PIP_ERR_WORKSPACE = -5
PIP_ERR_CUDA = -6
PIP_ERR_INVALID = -7
PIP_NOALLOC_MAX_POLYS = 65536


class PipStats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_uint64),
                ("bbox_rejects", ctypes.c_uint64),
                ("fallback_points", ctypes.c_uint64),
                ("exact_candidates", ctypes.c_uint64),
                ("filter_errors", ctypes.c_uint64),
                ("verified_pairs", ctypes.c_uint64),
                ("wait_timeouts", ctypes.c_uint64)]


class PipError(RuntimeError):
    def __init__(self, fn, code, lib=None):
        msg = f"{fn} returned {code}"
        if lib is not None:
            msg += ": " + lib.pip_status_str(code).decode()
            if code == PIP_ERR_CUDA:
                msg += f" (cudaError {lib.pip_last_cuda_error()})"
        super().__init__(msg)
        self.code = code


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_SIGS = {
    "pip_classify": ([_P, _I64, _P, _P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "pip_classify_exact": ([_P, _I64, _P, _P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "pip_classify_noalloc": ([_P, _I64, _P, _P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "pip_classify_paper": ([_P, _I64, _P, _P, _I32, _P, _P, _I32, _P, _P], ctypes.c_int),
    "pip_classify_slab": ([_P, _I64, _P, _P, _I32, _P, _P, _P, _P, _P], ctypes.c_int),
    "pip_slab_index_bytes": ([_I32, _I64, _I32, _I64], ctypes.c_size_t),
    "pip_quantize_lonlat": ([_P, _I64, ctypes.c_double, _P, _P, _P], ctypes.c_int),
    "pip_slab_build": ([_P, _P, _I32, _I64, _I32, _P, ctypes.c_size_t, _P, _P], ctypes.c_int),
    "pip_bin_workspace_bytes": ([_I64, _I32], ctypes.c_size_t),
    "pip_bin_index_bytes": ([_I32], ctypes.c_size_t),
    "pip_bin_index": ([_P, _P, _I32, _I32, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "pip_bin_probe_bytes": ([_I64, _I32], ctypes.c_size_t),
    "pip_bin_probe_count": ([_P, _I64, _P, ctypes.c_size_t, _I32, _P, ctypes.c_size_t, _P, _P, _P], ctypes.c_int),
    "pip_bin_probe_fill": ([_P, _I64, _P, ctypes.c_size_t, _I32, _P, ctypes.c_size_t, _P, _P, _I64, _P, _P],
                           ctypes.c_int),
    "pip_bin_count": ([_P, _I64, _P, _P, _I32, _I32, _P, ctypes.c_size_t, _P, _P, _P], ctypes.c_int),
    "pip_bin_fill": ([_P, _I64, _P, _P, _I32, _P, ctypes.c_size_t, _P, _P, _I64, _P, _P], ctypes.c_int),
    "pip_set_tuning": ([_I32, _I32, _I32], ctypes.c_int),
    "pip_get_tuning": ([_P, _P, _P], ctypes.c_int),
    "pip_set_small_tuning": ([_I32, _I32, _I32], ctypes.c_int),
    "pip_get_small_tuning": ([_P, _P, _P], ctypes.c_int),
    "pip_get_stats": ([ctypes.POINTER(PipStats)], ctypes.c_int),
    "pip_reset_stats": ([], ctypes.c_int),
    "pip_validate": ([_P, _I64, _P, _P, _I32, _I64, _P, _P, _I64, _P, _P], ctypes.c_int),
    "pip_status_str": ([ctypes.c_int], ctypes.c_char_p),
    "pip_last_cuda_error": ([], ctypes.c_int),
    "pip_version": ([], ctypes.c_int),
    "pip_launch_count": ([], ctypes.c_uint64),
    "pip_set_verify": ([_I32], ctypes.c_int),
    "pip_xor_words": ([_P, _P, _I64, _P], ctypes.c_int),
}


def load(path: str = LIB_PATH):
    """Open libpip.so (built by ``__graft_entry__.build()``) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libpip.so is not built ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def check(fn: str, code: int):
    if code != PIP_OK:
        raise PipError(fn, code, _lib)
    return code
