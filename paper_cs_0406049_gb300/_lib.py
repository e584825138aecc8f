"""ctypes loader for ``libsincos_gb300.so`` (the C ABI in include/sincos_pairs.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  If the library has not been built, loading fails loudly; there
is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsincos_gb300.so")

OK, EINVAL, EOVERLAP, ECUDA, EUNSUPPORTED, ECAPTURE = 0, -1, -2, -3, -4, -5
F32, BF16, F16 = 0, 1, 2
RED_PLAIN, RED_COMPENSATED = 0, 1
COEF_NORMALIZED, COEF_DAGGER = 0, 1
OP_PAIRS, OP_BACKWARD, OP_BATCHED, OP_EXPI, OP_HUYGENS = 0, 1, 2, 3, 4
NOALLOC_MAX_SEGMENTS = 65536
HOST_PATH_NONE, HOST_PATH_ZERO_COPY, HOST_PATH_PIPELINE, HOST_PATH_ZERO_COPY_PAGEABLE = 0, 1, 2, 3
HOST_ROUTE_AUTO, HOST_ROUTE_PIPELINE = 0, 1


class sincos_plan(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("unroll", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("vec_bytes", ctypes.c_int)]

    def as_dict(self):
        return {"block": self.block, "unroll": self.unroll, "ctas_per_sm": self.ctas_per_sm,
                "vec_bytes": self.vec_bytes}


class sincos_seg(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("s", ctypes.c_void_p), ("c", ctypes.c_void_p)]


# name -> (restype, argtypes); every symbol the header declares.
_VP, _I64, _INT, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
_PLANP = ctypes.POINTER(sincos_plan)
SIGNATURES = {
    "sincos_pairs": (_INT, [_VP, _VP, _VP, _I64, _VP]),
    "sincos_pairs_ex": (_INT, [_VP, _VP, _VP, _I64, _INT, _INT, _INT, _VP]),
    "sincos_expi": (_INT, [_VP, _VP, _I64, _INT, _INT, _VP]),
    "sincos_backward": (_INT, [_VP, _VP, _VP, _VP, _VP, _I64, _VP]),
    "sincos_huygens": (_INT, [_VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP, _I64, ctypes.c_float,
                              _INT, _VP, _VP]),
    "sincos_batched": (_INT, [_VP, _VP, _INT, _VP]),
    "sincos_batched_ex": (_INT, [_VP, _VP, _INT, _INT, _INT, _INT, _VP]),
    "sincos_batched_release": (_INT, []),
    "sincos_batched_noalloc": (_INT, [_VP, _VP, _INT, _INT, _INT, _INT, _VP]),
    "sincos_batched_graph_create": (_INT, [_VP, _VP, _INT, _INT, _INT, _INT,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "sincos_batched_graph_launch": (_INT, [_VP, _VP]),
    "sincos_batched_graph_destroy": (_INT, [_VP]),
    "sincos_pairs_host": (_INT, [_VP, _VP, _VP, _I64, _INT, _INT, _INT, _VP, _SZ, _VP]),
    "sincos_host_workspace_bytes": (_SZ, [_INT, _I64]),
    "sincos_host_last_path": (_INT, []),
    "sincos_host_route_set": (_INT, [_INT]),
    "sincos_plan_get": (_INT, [_INT, _INT, _I64, _PLANP]),
    "sincos_plan_set": (_INT, [_INT, _INT, _I64, _PLANP]),
    "sincos_autotune_pairs": (_INT, [_VP, _VP, _VP, _I64, _INT, _INT, _INT, _VP, _PLANP]),
    "sincos_autotune_backward": (_INT, [_VP, _VP, _VP, _VP, _VP, _I64, _VP, _PLANP]),
    "sincos_autotune_expi": (_INT, [_VP, _VP, _I64, _INT, _INT, _VP, _PLANP]),
    "sincos_autotune_huygens": (_INT, [_VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP, _I64,
                                       ctypes.c_float, _INT, _VP, _VP, _PLANP]),
    "sincos_autotune_batched": (_INT, [_VP, _VP, _INT, _INT, _INT, _INT, _VP, _PLANP]),
    "sincos_plan_cache_save": (_INT, [ctypes.c_char_p]),
    "sincos_plan_cache_load": (_INT, [ctypes.c_char_p]),
    "sincos_strerror": (ctypes.c_char_p, [_INT]),
    "sincos_last_error": (ctypes.c_char_p, []),
    "sincos_device_wait_timeouts": (ctypes.c_uint32, []),
    "sincos_device_bad_segments": (ctypes.c_uint32, []),
    "sincos_seg_check": (_INT, [ctypes.c_void_p, _I64, _INT]),
    "sincos_selftest_wait_timeout": (_INT, [ctypes.c_uint32, _VP]),
    "sincos_launch_count": (ctypes.c_uint64, []),
    "sincos_version": (_INT, []),
}

_lock = threading.Lock()
_lib = None


class SincosError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        lib = _lib
        detail = ""
        if lib is not None:
            detail = lib.sincos_strerror(status).decode()
            if status == ECUDA:
                detail += ": " + lib.sincos_last_error().decode()
        super().__init__(f"{what} failed with status {status} ({detail})")


def load(path: str = LIB_PATH):
    """Load the library (once) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()'). "
                "There is no CPU fallback.")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, what: str) -> None:
    if status != OK:
        raise SincosError(status, what)
